// api.cu -- C ABI of libmotjvie (declared in include/motjvie.h) and the host
// orchestration of the device passes: Galerkin tables and spectra, the
// matrix-free Z0 product (Eq. 11-12), the history right-hand side (Eq. 3),
// the TFQMR solve of each step and the history ring.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/motjvie.h"
#include "common.cuh"
#include "fft.cuh"
#include "galerkin.cuh"
#include "krylov.cuh"
#include "spectral.cuh"
#include "tables.cuh"
#include "peak.cuh"
#include "direct.cuh"

#include <atomic>
#include <memory>
#include <chrono>
#include <mutex>

namespace mot {
static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void set_error(const std::string &msg) { g_err = msg; }
const char *get_error() { return g_err.c_str(); }
}  // namespace mot

using namespace mot;

#define MOT_FAIL(code, msg)          \
    do {                             \
        ::mot::set_error(msg);       \
        return code;                 \
    } while (0)

#define MOT_CHECK_LAUNCH() MOT_CUDA_TRY(cudaGetLastError())

#define MOT_TRY(...)                      \
    do {                                  \
        mot_status _s = (__VA_ARGS__);    \
        if (_s != MOT_OK) return _s;      \
    } while (0)

namespace {

constexpr double kC0 = 299792458.0;

// ---------------------------------------------------------------- device memory
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

mot_status dalloc(DBuf &b, size_t bytes) {
    if (b.bytes >= bytes && b.p) return MOT_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (bytes == 0) return MOT_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        return MOT_ENOMEM;
    }
    b.bytes = bytes;
    return MOT_OK;
}

void dfree(DBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int grid_for(long n, int threads = 256) {
    long g = (n + threads - 1) / threads;
    if (g > 148 * 16) g = 148 * 16;
    if (g < 1) g = 1;
    return (int)g;
}

// ---------------------------------------------------------------- Gauss-Legendre (host)
void gauss_legendre(int n, double *x, double *w) {
    const double pi = 3.141592653589793238462643383279502884;
    for (int i = 0; i < n; ++i) {
        double z = cos(pi * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 200; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) <= 1e-16) break;
        }
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

constexpr int kGLN = 20;  // radial panels
constexpr int kGL8 = 8;   // z-line pieces far from the origin

// the kGLN-point rule followed by the kGL8-point rule
struct HostRule {
    double x[kGLN + kGL8], w[kGLN + kGL8];
    HostRule() {
        gauss_legendre(kGLN, x, w);
        gauss_legendre(kGL8, x + kGLN, w + kGLN);
    }
};
const HostRule &host_rule() {
    static HostRule r;
    return r;
}

// ---------------------------------------------------------------- table items
// sorted offsets (a <= b <= c) that fit the sorted extents S and the lags in
// [k0, k1] whose causal support contains them, enumerated offset-major; the
// sorted offsets' box-integral records and the distinct plane integrals their
// diagonal entries need (knot-interval moments, see galerkin.cuh).
struct ItemSet {
    std::vector<TableItem> items;
    std::vector<int> base, klo, cnt;  // per dense triple index (Rm+1)^3
    int Rm = 0;
    std::vector<TripleRec> tri;
    std::vector<FaceRec> faces;
    long fm_len = 0, bm_len = 0;  // doubles of face / box moments
};

// false: a support meets more knot intervals than one record holds (rho < 0.25)
bool build_items(double rho, const int S[3], int k0, int k1, ItemSet &is) {
    int Rm = S[2];
    is.Rm = Rm;
    long n3 = (long)(Rm + 1) * (Rm + 1) * (Rm + 1);
    is.base.assign(n3, -1);
    is.klo.assign(n3, 0);
    is.cnt.assign(n3, 0);
    is.items.clear();
    is.tri.clear();
    is.faces.clear();
    is.fm_len = is.bm_len = 0;
    const int jg0 = std::max(0, k0 - 2), jg1 = k1;
    // distinct faces (c, a <= b), c in [0, Rm + 1], a, b in [0, Rm]
    const long fkeys = (long)(Rm + 2) * (Rm + 1) * (Rm + 1);
    std::vector<int> fid(fkeys, -1);
    auto face_of = [&](int c, int a, int b) -> int {
        c = std::abs(c);
        a = std::abs(a);
        b = std::abs(b);
        if (a > b) std::swap(a, b);
        const long key = ((long)c * (Rm + 1) + a) * (Rm + 1) + b;
        int &id = fid[key];
        if (id >= 0) return id;
        FaceRec f = {c, a, b, 0, 0, is.fm_len};
        const double lo2 = std::pow(std::max(a - 1.0, 0.0), 2) + std::pow(std::max(b - 1.0, 0.0), 2);
        const double hi2 = std::pow(a + 1.0, 2) + std::pow(b + 1.0, 2);
        if (gk::interval_range(rho, sqrt((double)c * c + lo2), sqrt((double)c * c + hi2), jg0, jg1, &f.jlo, &f.nj))
            is.fm_len += 3L * f.nj;
        else
            f.nj = 0;
        id = (int)is.faces.size();
        is.faces.push_back(f);
        return id;
    };
    for (int a = 0; a <= S[0]; ++a)
        for (int b = a; b <= S[1]; ++b)
            for (int c = b; c <= S[2]; ++c) {
                double lo = 0.0, hi = 0.0;
                int d[3] = {a, b, c};
                for (int i = 0; i < 3; ++i) {
                    double l = std::max(d[i] - 1.0, 0.0), h = d[i] + 1.0;
                    lo += l * l;
                    hi += h * h;
                }
                lo = sqrt(lo);
                hi = sqrt(hi);
                int kb = std::max(k0, (int)floor(lo / rho - 1.0) - 1);
                int ke = std::min(k1, (int)ceil(hi / rho + 2.0) + 1);
                long key = ((long)a * (Rm + 1) + b) * (Rm + 1) + c;
                int first = -1, count = 0, kfirst = 0;
                for (int k = kb; k <= ke; ++k) {
                    if (!gk::support(k, rho, a, b, c)) continue;
                    if (first < 0) {
                        first = (int)is.items.size();
                        kfirst = k;
                        TripleRec t;
                        t.x = a;
                        t.y = b;
                        t.z = c;
                        t.off = is.bm_len;
                        if (gk::interval_range(rho, lo, hi, jg0, jg1, &t.jlo, &t.nj)) {
                            if (t.nj > gk::kMaxIntervals) return false;
                            is.bm_len += 9L * t.nj;
                        } else {
                            t.jlo = 0;
                            t.nj = 0;
                        }
                        for (int p = 0; p < 3; ++p)
                            for (int e = -1; e <= 1; ++e)
                                t.face[3 * p + e + 1] = face_of(d[p] + e, d[(p + 1) % 3], d[(p + 2) % 3]);
                        is.tri.push_back(t);
                    }
                    // lags of one offset form a contiguous range
                    is.items.push_back({k, a, b, c, (int)is.tri.size() - 1});
                    ++count;
                }
                if (first >= 0) {
                    is.base[key] = first;
                    is.klo[key] = kfirst;
                    is.cnt[key] = count;
                }
            }
    for (const FaceRec &f : is.faces)
        if (f.nj > gk::kMaxIntervals) return false;
    return true;
}

// process-wide cache of quadrature results: the lag tables depend only on
// rho, the table extents and the lag range (not on eps_r), so problems that
// share them reuse the A values instead of recomputing the quadrature
struct TableCacheEntry {
    double rho;
    int S[3], k0, k1;
    std::vector<double> A6;
    // the per-offset item ranges of the item set (what a cached set-up needs of it)
    int Rm = 0;
    std::vector<int> base, klo, cnt;
};
std::mutex g_tcache_mu;
std::vector<std::shared_ptr<const TableCacheEntry>> g_tcache;
constexpr size_t kTableCacheEntries = 8;

std::shared_ptr<const TableCacheEntry> tcache_find(double rho, const int S[3], int k0, int k1) {
    std::lock_guard<std::mutex> lk(g_tcache_mu);
    for (auto &e : g_tcache)
        if (e->rho == rho && e->S[0] == S[0] && e->S[1] == S[1] && e->S[2] == S[2] && e->k0 == k0 && e->k1 == k1)
            return e;
    return nullptr;
}

void tcache_put(double rho, const int S[3], int k0, int k1, std::vector<double> &&A6, const ItemSet &is) {
    auto e = std::make_shared<TableCacheEntry>();
    e->rho = rho;
    for (int i = 0; i < 3; ++i) e->S[i] = S[i];
    e->k0 = k0;
    e->k1 = k1;
    e->A6 = std::move(A6);
    e->Rm = is.Rm;
    e->base = is.base;
    e->klo = is.klo;
    e->cnt = is.cnt;
    std::lock_guard<std::mutex> lk(g_tcache_mu);
    if (g_tcache.size() >= kTableCacheEntries) g_tcache.erase(g_tcache.begin());
    g_tcache.push_back(std::move(e));
}

// per-lag map triple -> item (or -1), from the offset-major ranges
void lag_map(const ItemSet &is, int k, std::vector<int> &map) {
    map.assign(is.base.size(), -1);
    for (size_t i = 0; i < is.base.size(); ++i)
        if (is.base[i] >= 0 && k >= is.klo[i] && k < is.klo[i] + is.cnt[i]) map[i] = is.base[i] + (k - is.klo[i]);
}

int lag_reach(int k, double rho) { return gk::reach(k, rho); }

// set-up phase timings on stderr when MOTJVIE_TRACE=1 (profiling the set-up)
struct PhaseTrace {
    const char *what;
    std::chrono::steady_clock::time_point t0;
    static bool on() {
        static const bool f = getenv("MOTJVIE_TRACE") && atoi(getenv("MOTJVIE_TRACE")) != 0;
        return f;
    }
    explicit PhaseTrace(const char *w) : what(w), t0(std::chrono::steady_clock::now()) {}
    ~PhaseTrace() {
        if (!on()) return;
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        fprintf(stderr, "[motjvie] %s: %.1f ms\n", what, ms);
    }
};

// cos / sin coefficient tables of one axis: [K][R+1]
void axis_coef(int M, int R, bool odd, std::vector<double> &cf) {
    const double pi = 3.141592653589793238462643383279502884;
    int K = M / 2 + 1;
    cf.assign((size_t)K * (R + 1), 0.0);
    for (int k = 0; k < K; ++k)
        for (int d = 0; d <= R; ++d) {
            long m = ((long)k * d) % M;
            double ang = 2.0 * pi * (double)m / (double)M;
            double v;
            if (odd) v = d == 0 ? 0.0 : 2.0 * sin(ang);
            else v = d == 0 ? 1.0 : 2.0 * cos(ang);
            cf[(size_t)k * (R + 1) + d] = v;
        }
}

}  // namespace

// ============================================================================
// handles
// ============================================================================
struct AxisTw {
    int M = 0;
    FftPlan plan{};    // FP32 passes
    FftPlan plan64{};  // FP64 and double-float passes (radix <= 9: register pressure)
    DBuf tw64, tw32, twdf;  // twiddles in FP64, FP32 and double-float (hi, lo pairs)
};

struct mot_ctx {
    int device = 0;
    int sms = 148;  // multiprocessors of the device
    cudaStream_t stream = nullptr;
    bool own_stream = false;
};

struct LagTable {
    DBuf oct;       // FP64 octant [6][Rz+1][Ry+1][Rx+1]
    int R[3] = {0, 0, 0};
    bool ready = false;
    bool override_ = false;
};

// event pairs around selected kernels (timing option)
struct KTimer {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> cls;
    int used = 0;
    void begin(cudaStream_t st, int c) {
        if (!on) return;
        if ((int)ev.size() < 2 * (used + 1)) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            ev.push_back(a);
            ev.push_back(b);
        }
        cls.resize(used + 1);
        cls[used] = c;
        cudaEventRecord(ev[2 * used], st);
    }
    void end(cudaStream_t st) {
        if (!on) return;
        cudaEventRecord(ev[2 * used + 1], st);
        ++used;
    }
    int count(int c) const {
        int k = 0;
        for (int i = 0; i < used; ++i) k += cls[i] == c;
        return k;
    }
    float total(int c) {
        float acc = 0.f;
        for (int i = 0; i < used; ++i)
            if (cls[i] == c) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
                acc += ms;
            }
        return acc;
    }
    void reset() { used = 0; }
    ~KTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

// ---------------------------------------------------------------- launch schedules
// Launch choices of the Z0 product that leave its arithmetic unchanged (every
// output element goes through the same operations in the same order whatever
// is picked): columns per z-pass block, rows per row-pass block, plane-pass
// block sizes of the plain product, programmatic dependent launch, and the row
// pairs / tile widths of the generic passes.  0 = the built-in rule.  The
// autotuner (tune_product) picks them per (grid, right-hand sides, precision);
// the product and the march launch under the schedule made current by a
// SchedScope.  The MOTJVIE_* environment switches, where set, override it.
struct Sched {
    int z_cols = 0;     // z-pass columns per block: 4 | 8 | 16 | 32
    int x_rows = 0;     // rows per block of the compiled row passes: 8 | 16 | 32
    int xy_fwd = 0;     // plane-pass block size of the plain product: 256 | 384 | 512
    int xy_inv = 0;
    int pdl = 1;        // programmatic dependent launch of the chain kernels
    int gen_pairs = 0;  // generic x passes: row pairs per block, 1..8
    int gen_tile = 0;   // generic axis passes: columns per block, power of two
    int z_tma = 0;      // z pass: stage the column tiles with TMA (cp.async.bulk.tensor) when 1
};
thread_local const Sched *t_sched = nullptr;
inline const Sched &cur_sched() {
    static const Sched d;
    return t_sched ? *t_sched : d;
}
struct SchedScope {
    const Sched *prev;
    explicit SchedScope(const Sched *s) : prev(t_sched) { t_sched = s; }
    ~SchedScope() { t_sched = prev; }
};

// device memory shared by problems (the history spectra of problems with the
// same step, grid and precision): freed with the last problem holding it
struct SharedDev {
    void *p = nullptr;
    size_t bytes = 0;
    int device = 0;
    ~SharedDev() {
        if (!p) return;
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        cudaFree(p);
        cudaSetDevice(cur);
    }
};

struct mot_problem {
    mot_ctx *ctx = nullptr;
    KTimer kt;
    bool capturing = false;
    int N[3];
    double h, alpha, rho, dt;
    int ell;
    int M0[3], Mh[3], H0, Hh;
    int K0[3], Kh[3];
    int r0;
    std::vector<double> eps_host;
    DBuf eps, eps32;  // eps_r in FP64 and FP32
    std::vector<AxisTw *> tws;
    std::vector<LagTable> lags;
    DBuf L0_64, L0_32, L0_df;  // [6][K0z][K0y][H0] in FP64, FP32, double-float
    DBuf Lh_64, Lh_32, Lh_df;  // [ell+1][6][Khz][Khy][Hh] in FP64, FP32, double-float
    std::shared_ptr<SharedDev> lh_hold[3];  // set when Lh_64 / Lh_32 / Lh_df is shared (not owned)
    bool hist64 = false, hist32 = false, histdf = false;
    DBuf glx, glw;
    // Z0 product workspace
    DBuf wsA, wsB;
    mot_options opt;
    // tuned launch schedules of the Z0 product, per (right-hand sides, FP32)
    struct Tuned {
        int nrhs, fp32;
        Sched s;
        mot_schedule info;
    };
    std::vector<Tuned> tuned;
    // TMA descriptors of the z pass, per planes buffer and shape
    struct ZMap {
        const void *ptr;
        long rows, ncols;
        int Nz, TC, es;
        CUtensorMap map;
    };
    std::vector<ZMap> zmaps;
    // the direct product's offset list of the lag-0 support (per precision and tile)
    struct DirectList {
        int fp32 = -1, SX = 0, SY = 0, nd = 0;
        DBuf d, g;
    } direct;
    const Sched *sched_for(int nrhs, bool fp32) const {
        for (auto &t : tuned)
            if (t.nrhs == nrhs && t.fp32 == (int)fp32) return &t.s;
        return nullptr;
    }
};

struct LoopGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *x = nullptr;
    int body_kernels = 0;
};

struct mot_run {
    mot_problem *p = nullptr;
    cudaStream_t cap = nullptr;  // capture stream for the solve graphs
    LoopGraph loop64, loop32;
    DBuf ctl;                    // device loop control: iteration count, cap, continue flag
    DBuf ctr;                    // last-block tickets of the fused TFQMR reduction kernels (0 between launches)
    DBuf inctab;                 // axis tables of the fast incident path
    int B = 1;
    int prec = MOT_FP64;
    long n = 0;  // next step index
    std::vector<PlaneWaveDev> pw_host;
    std::vector<mot_planewave> exc_host;  // the plane waves as given (checkpoints)
    bool warmed = false;  // one host-driven step done in this process (graph mode needs it first)
    DBuf pw, inc, J, J2, J3, b, r;  // J2, J3: J_{n-2}, J_{n-3} for the extrapolated guesses (J3: guess 2 only)
    DBuf ring, wsAh, wsBh;
    DBuf hacc;  // history accumulation on the full Mh grid [B][3][Mhz][Mhy][Hh]
    // time-blocked history: the lags 2.. partial sums of the steps of the current
    // time block, 2 hTB rotating slots of hacc's layout (slot m mod 2 hTB): the
    // current block's partial sums and the next block's, filled beside this block's steps
    DBuf hpart;
    int hTB = 8;
    bool hpart_ok = false;  // the slot of step n holds its whole lags 2.. sum (the step graph leaves it so)
    bool q_stale = true;    // the slots hold nothing usable (a new run, a loaded checkpoint): rebuild from the block start
    cudaStream_t hside = nullptr;  // step graph: side branch of the next step's partial sum
    cudaEvent_t hfork = nullptr, hjoin = nullptr;
    bool hjoin_open = false;  // capture: the branch still has to join the step's stream
    // Krylov vectors (type of the solve) and scratch
    DBuf kv[10];
    DBuf scal, part1, part2, part3, dots;
    DBuf r32;  // mixed: residual in FP32 / correction
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> sev;  // graph mode: start/end event of each step of a chunk
    // graph mode with J_out: J_n is copied on the device into one of two staging
    // buffers and from there to the host on its own stream, beside the next step
    DBuf jstage[2];
    cudaStream_t jcopy = nullptr;
    cudaEvent_t jready[2] = {nullptr, nullptr}, jdone[2] = {nullptr, nullptr};
    // whole-step graph (graph mode)
    cudaStream_t cap2 = nullptr, cap3 = nullptr;
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    DBuf sdev;      // StepDev
    DBuf sstats;    // per-step device stats of one mot_run_step call
    DBuf b2, r2;    // ||b||^2, ||r||^2 per right-hand side
    int sstats_cap = 0;
    int k_fixed = 0, k_outer = 0, k_inner = 0;  // kernels per step / per sweep / per TFQMR iteration
};

namespace {

AxisTw *get_tw(mot_problem *p, int M) {
    for (auto *t : p->tws)
        if (t->M == M) return t;
    AxisTw *t = new AxisTw();
    t->M = M;
    // largest register radix of the FP32 passes (tuning knob, default 16)
    int max_radix = 16;
    if (const char *ev = getenv("MOTJVIE_MAX_RADIX")) max_radix = std::max(2, atoi(ev));
    if (!make_plan(M, &t->plan, max_radix) || !make_plan(M, &t->plan64, std::min(max_radix, 9))) {
        delete t;
        return nullptr;
    }
    std::vector<double2> h64(M);
    std::vector<float2> h32(M);
    std::vector<float4> hdf(M);  // (re.hi, re.lo, im.hi, im.lo)
    const double pi = 3.141592653589793238462643383279502884;
    for (int m = 0; m < M; ++m) {
        double a = -2.0 * pi * (double)m / (double)M;
        h64[m] = make_double2(cos(a), sin(a));
        h32[m] = make_float2((float)cos(a), (float)sin(a));
        const float ch = (float)cos(a), sh = (float)sin(a);
        hdf[m] = make_float4(ch, (float)(cos(a) - (double)ch), sh, (float)(sin(a) - (double)sh));
    }
    if (dalloc(t->tw64, sizeof(double2) * M) != MOT_OK || dalloc(t->tw32, sizeof(float2) * M) != MOT_OK ||
        dalloc(t->twdf, sizeof(float4) * M) != MOT_OK) {
        delete t;
        return nullptr;
    }
    cudaMemcpy(t->tw64.p, h64.data(), sizeof(double2) * M, cudaMemcpyHostToDevice);
    cudaMemcpy(t->tw32.p, h32.data(), sizeof(float2) * M, cudaMemcpyHostToDevice);
    cudaMemcpy(t->twdf.p, hdf.data(), sizeof(float4) * M, cudaMemcpyHostToDevice);
    p->tws.push_back(t);
    return t;
}

template <typename T> const FftPlan &planp(AxisTw *t);
template <> const FftPlan &planp<double>(AxisTw *t) { return t->plan64; }
template <> const FftPlan &planp<float>(AxisTw *t) { return t->plan; }
template <> const FftPlan &planp<dfl>(AxisTw *t) { return t->plan64; }

template <typename T> const cplx<T> *twp(AxisTw *t);
template <> const cplx<double> *twp<double>(AxisTw *t) { return (const double2 *)t->tw64.p; }
template <> const cplx<float> *twp<float>(AxisTw *t) { return (const float2 *)t->tw32.p; }
template <> const cplx<dfl> *twp<dfl>(AxisTw *t) { return (const dfl2 *)t->twdf.p; }

constexpr size_t kSmemMax = 200 * 1024;
// block sizes: the pencil passes are latency-bound at small grids, so they use
// large CTAs to keep enough warps resident
constexpr int kZThreads = 512;

// raise the dynamic shared-memory limit of one kernel, once per kernel
template <auto Kern> mot_status allow_smem() {
    static bool done = false;
    if (!done) {
        MOT_CUDA_TRY(cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax));
        done = true;
    }
    return MOT_OK;
}

// ---------------------------------------------------------------- pass launchers
template <typename TI, typename T>
mot_status launch_x_forward(const TI *x, cplx<T> *out, long nrows, int Nx, int H, AxisTw *tw, cudaStream_t st) {
    const int M = tw->M;
    int pairs = (int)std::min<long>(8, std::max<long>(1, ((long)(48 * 1024) / ((long)M * sizeof(cplx<T>)) - 1) / 2));
    const int sp = cur_sched().gen_pairs;
    if (sp >= 1 && sp <= 8 && (size_t)(2 * sp + 1) * M * sizeof(cplx<T>) <= kSmemMax) pairs = sp;
    size_t smem = (size_t)(2 * pairs + 1) * M * sizeof(cplx<T>);
    MOT_TRY(allow_smem<k_x_forward<TI, T>>());
    long grid = (nrows + 2 * pairs - 1) / (2 * pairs);
    count_launch();
    k_x_forward<TI, T><<<(unsigned)grid, 256, smem, st>>>(x, out, nrows, Nx, H, planp<T>(tw), twp<T>(tw), pairs);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

template <typename T> int tile_width(int M, int comps) {
    int tx = comps > 1 ? (sizeof(T) == 4 ? 8 : 4) : (sizeof(T) == 4 ? 16 : 8);
    while (tx > 1 && (size_t)(2 * comps * M * tx + M) * sizeof(cplx<T>) > kSmemMax) tx /= 2;
    return tx;
}

template <typename T, int S>
mot_status launch_axis(const cplx<T> *in, cplx<T> *out, AxisTw *tw, int H, int Lin, int Lout, int O1, int O2,
                       long is1, long is2, long ias, long os1, long os2, long oas, cudaStream_t st,
                       const long long *nptr = nullptr, int ell = 1, long slot_stride = 0) {
    const int M = tw->M;
    int tx = tile_width<T>(M, 1);
    const int st_ = cur_sched().gen_tile;
    if (st_ >= 1 && st_ < tx && (st_ & (st_ - 1)) == 0) tx = st_;
    size_t smem = (size_t)(2 * M * tx + M) * sizeof(cplx<T>);
    MOT_TRY(allow_smem<k_axis<T, S>>());
    dim3 grid((H + tx - 1) / tx, (unsigned)(O1 * O2));
    count_launch();
    k_axis<T, S><<<grid, kZThreads, smem, st>>>(in, out, planp<T>(tw), twp<T>(tw), H, tx, Lin, Lout, O2, is1, is2, ias, os1,
                                          os2, oas, nptr, ell, slot_stride);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

template <typename T, class Epi>
mot_status launch_x_inverse(const cplx<T> *in, long nrows, int Nx, int H, AxisTw *tw, Epi epi, cudaStream_t st) {
    const int M = tw->M;
    int pairs = (int)std::min<long>(8, std::max<long>(1, (long)(64 * 1024) / ((long)(2 * H + 2 * M + M) * sizeof(cplx<T>))));
    const int sp = cur_sched().gen_pairs;
    if (sp >= 1 && sp <= 8 && (size_t)(2 * sp * H + 2 * sp * M + M) * sizeof(cplx<T>) <= kSmemMax) pairs = sp;
    size_t smem = (size_t)(2 * pairs * H + 2 * pairs * M + M) * sizeof(cplx<T>);
    MOT_TRY(allow_smem<k_x_inverse<T, Epi>>());
    long grid = (nrows + 2 * pairs - 1) / (2 * pairs);
    count_launch();
    k_x_inverse<T, Epi><<<(unsigned)grid, 256, smem, st>>>(in, nrows, Nx, H, planp<T>(tw), twp<T>(tw), pairs, epi);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

// the chain kernels of a Z0 product (plane passes, z pass) go out with
// programmatic dependent launch: the next kernel's blocks start while the
// previous kernel finishes (its last blocks and its reduction tail) and wait on
// the device; MOTJVIE_PDL=0 turns it off (timing comparisons)
inline bool chain_pdl_on() {
    static const bool off = getenv("MOTJVIE_PDL") && atoi(getenv("MOTJVIE_PDL")) == 0;
    return !off && cur_sched().pdl != 0;
}
template <typename... KArgs, typename... Args>
void launch_chain(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    if (!chain_pdl_on()) {
        kern<<<grid, block, smem, st>>>(args...);
        return;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);  // an error stays the last error, checked by the caller
}

// threads of a specialised plane-pass block.  512 threads shorten each stage
// with few planes (one right-hand side: about one block per SM) and suit the
// vector-heavy solver passes (the FP64 residual epilogue at 16 right-hand
// sides: 162 us at 512 threads, 231 us at 384).  The plain FP32 product with
// many waves of planes runs faster in smaller blocks, more of them resident
// and fewer threads idle at the stage barriers (72^2 planes, 16 right-hand
// sides: forward 53.4 / 50.5 / 44.8 us and inverse 56.1 / 51.4 / 55.0 us at
// 512 / 384 / 256 threads).  MOTJVIE_XY_THREADS = 256 | 384 | 512 overrides,
// for timing sweeps.
inline int sm_count() {
    static const int n = [] {
        int dev = 0, v = 148;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v;
    }();
    return n;
}
inline int xy_threads(int planes, bool forward, bool plain32) {
    static const int f = getenv("MOTJVIE_XY_THREADS") ? atoi(getenv("MOTJVIE_XY_THREADS")) : 0;
    if (f == 256 || f == 384 || f == 512) return f;
    if (!plain32) return 512;
    const int s = forward ? cur_sched().xy_fwd : cur_sched().xy_inv;
    if (s == 256 || s == 384 || s == 512) return s;
    if (planes < 4 * sm_count()) return 512;
    return forward ? 256 : 384;
}

// specialised plane kernels for the compiled (Mx, My) shapes; false -> generic
template <class Src, typename T, int RX1, int RX2, int RY1, int RY2>
bool xy_forward_r_go(Src x, cplx<T> *out, int planes, int Nx, int Ny, AxisTw *tx, AxisTw *ty, cudaStream_t st) {
    const size_t smem = xy_r_smem_bytes<T, RX1, RX2, RY1, RY2>(Ny);
    if (smem > kSmemMax) return false;
    if (allow_smem<k_xy_forward_r<Src, T, RX1, RX2, RY1, RY2>>() != MOT_OK) return false;
    count_launch();
    launch_chain(k_xy_forward_r<Src, T, RX1, RX2, RY1, RY2>, dim3(planes),
                 dim3(xy_threads(planes, true, std::is_same<Src, SrcPlain<float>>::value && sizeof(T) == 4)), smem, st,
                 x, out, Nx, Ny,
                 twp<T>(tx), twp<T>(ty));
    return true;
}

template <typename T, class Epi, int RX1, int RX2, int RY1, int RY2>
bool xy_inverse_r_go(const cplx<T> *in, int planes, int Nx, int Ny, int Nz, AxisTw *tx, AxisTw *ty, Epi epi,
                     cudaStream_t st) {
    const size_t smem = xy_r_smem_bytes<T, RX1, RX2, RY1, RY2>(Ny);
    if (smem > kSmemMax) return false;
    if (allow_smem<k_xy_inverse_r<T, Epi, RX1, RX2, RY1, RY2>>() != MOT_OK) return false;
    count_launch();
    launch_chain(k_xy_inverse_r<T, Epi, RX1, RX2, RY1, RY2>, dim3(planes),
                 dim3(xy_threads(planes, false, std::is_same<Epi, EpiZ0<float, float>>::value)), smem, st, in, Nx, Ny, Nz,
                 twp<T>(tx), twp<T>(ty), epi);
    return true;
}

inline bool specialised_off() {
    static const bool off = getenv("MOTJVIE_GENERIC_FFT") && atoi(getenv("MOTJVIE_GENERIC_FFT")) != 0;
    return off;
}

template <class Src, typename T>
bool xy_forward_r(Src x, cplx<T> *out, int planes, int Nx, int Ny, AxisTw *tx, AxisTw *ty, cudaStream_t st) {
    if (specialised_off() || tx->M != ty->M) return false;
    switch (tx->M) {
        case 20: return xy_forward_r_go<Src, T, 5, 4, 5, 4>(x, out, planes, Nx, Ny, tx, ty, st);
        case 32: return xy_forward_r_go<Src, T, 8, 4, 8, 4>(x, out, planes, Nx, Ny, tx, ty, st);
        case 72: return xy_forward_r_go<Src, T, 9, 8, 9, 8>(x, out, planes, Nx, Ny, tx, ty, st);
        case 75: return xy_forward_r_go<Src, T, 5, 15, 5, 15>(x, out, planes, Nx, Ny, tx, ty, st);
        case 128: return xy_forward_r_go<Src, T, 16, 8, 16, 8>(x, out, planes, Nx, Ny, tx, ty, st);
        default: return false;
    }
}

template <typename T, class Epi>
bool xy_inverse_r(const cplx<T> *in, int planes, int Nx, int Ny, int Nz, AxisTw *tx, AxisTw *ty, Epi epi, cudaStream_t st) {
    if (specialised_off() || tx->M != ty->M) return false;
    switch (tx->M) {
        case 20: return xy_inverse_r_go<T, Epi, 5, 4, 5, 4>(in, planes, Nx, Ny, Nz, tx, ty, epi, st);
        case 32: return xy_inverse_r_go<T, Epi, 8, 4, 8, 4>(in, planes, Nx, Ny, Nz, tx, ty, epi, st);
        case 72: return xy_inverse_r_go<T, Epi, 9, 8, 9, 8>(in, planes, Nx, Ny, Nz, tx, ty, epi, st);
        case 75: return xy_inverse_r_go<T, Epi, 5, 15, 5, 15>(in, planes, Nx, Ny, Nz, tx, ty, epi, st);
        case 128: return xy_inverse_r_go<T, Epi, 16, 8, 16, 8>(in, planes, Nx, Ny, Nz, tx, ty, epi, st);
        default: return false;
    }
}

// specialised row / column passes for the compiled lengths of planes too
// large for shared memory; false -> generic
template <typename TI, typename T, int R1, int R2, int P>
bool x_forward_r_go(const TI *x, cplx<T> *out, long nrows, int Nx, AxisTw *tw, cudaStream_t st) {
    constexpr size_t smem = x_r_smem<T, R1, R2, P>();
    if (smem > kSmemMax || allow_smem<k_x_forward_r<TI, T, R1, R2, P>>() != MOT_OK) return false;
    count_launch();
    launch_chain(k_x_forward_r<TI, T, R1, R2, P>, dim3((unsigned)(nrows / (2 * P))), dim3(P * R2), smem, st, x, out,
                 Nx, twp<T>(tw));
    return true;
}

template <typename T, class Epi, int R1, int R2, int P>
bool x_inverse_r_go(const cplx<T> *in, long nrows, int Nx, int Ny, int Nz, AxisTw *tw, Epi epi, cudaStream_t st) {
    constexpr size_t smem = x_r_smem<T, R1, R2, P>();
    if (smem > kSmemMax || allow_smem<k_x_inverse_r<T, Epi, R1, R2, P>>() != MOT_OK) return false;
    count_launch();
    launch_chain(k_x_inverse_r<T, Epi, R1, R2, P>, dim3((unsigned)(nrows / (2 * P))), dim3(P * R2), smem, st, in, Nx,
                 Ny, Nz, twp<T>(tw), epi);
    return true;
}

template <typename T, int S, int R1, int R2, int TC>
bool col_r_go(const cplx<T> *in, cplx<T> *out, AxisTw *tw, int H, int Lin, int Lout, int planes, long ips, long ops,
              cudaStream_t st, const long long *nptr, int ell, long slot_stride) {
    constexpr int M = R1 * R2;
    const size_t smem = (size_t)(M + TC * (M + 1)) * sizeof(cplx<T>);
    if (smem > kSmemMax || allow_smem<k_col_r<T, S, R1, R2, TC>>() != MOT_OK) return false;
    count_launch();
    launch_chain(k_col_r<T, S, R1, R2, TC>, dim3((H + TC - 1) / TC, planes), dim3(TC * R2), smem, st, in, out,
                 twp<T>(tw), H, Lin, Lout, ips, ops, nptr, ell, slot_stride);
    return true;
}

// rows per block 2P: the schedule's choice where it divides Ny, else the
// largest of 32, 16, 8 dividing Ny (blocks stay inside one plane)
inline int x_rows_for(int Ny) {
    const int s = cur_sched().x_rows;
    if ((s == 8 || s == 16 || s == 32) && Ny % s == 0) return s;
    for (int r : {32, 16, 8})
        if (Ny % r == 0) return r;
    return 0;
}

template <typename TI, typename T>
bool x_forward_r(const TI *x, cplx<T> *out, long nrows, int Nx, int Ny, AxisTw *tw, cudaStream_t st) {
    if (specialised_off()) return false;
    switch (tw->M) {
        case 270:
            switch (x_rows_for(Ny)) {
                case 32: return x_forward_r_go<TI, T, 15, 18, 16>(x, out, nrows, Nx, tw, st);
                case 16: return x_forward_r_go<TI, T, 15, 18, 8>(x, out, nrows, Nx, tw, st);
                case 8: return x_forward_r_go<TI, T, 15, 18, 4>(x, out, nrows, Nx, tw, st);
                default: return false;
            }
        case 512:  // the history grid of the 256 x 256 pillar array: 16 x 32, four row pairs per block
            return Ny % 8 == 0 && x_forward_r_go<TI, T, 16, 32, 4>(x, out, nrows, Nx, tw, st);
        default: return false;
    }
}

template <typename T, class Epi>
bool x_inverse_r(const cplx<T> *in, long nrows, int Nx, int Ny, int Nz, AxisTw *tw, Epi epi, cudaStream_t st) {
    if (specialised_off()) return false;
    switch (tw->M) {
        case 270:
            switch (x_rows_for(Ny)) {
                case 32: return x_inverse_r_go<T, Epi, 15, 18, 16>(in, nrows, Nx, Ny, Nz, tw, epi, st);
                case 16: return x_inverse_r_go<T, Epi, 15, 18, 8>(in, nrows, Nx, Ny, Nz, tw, epi, st);
                case 8: return x_inverse_r_go<T, Epi, 15, 18, 4>(in, nrows, Nx, Ny, Nz, tw, epi, st);
                default: return false;
            }
        case 512:
            return Ny % 8 == 0 && x_inverse_r_go<T, Epi, 16, 32, 4>(in, nrows, Nx, Ny, Nz, tw, epi, st);
        default: return false;
    }
}

template <typename T, int S>
bool col_r(const cplx<T> *in, cplx<T> *out, AxisTw *tw, int H, int Lin, int Lout, int planes, long ips, long ops,
           cudaStream_t st, const long long *nptr = nullptr, int ell = 1, long slot_stride = 0) {
    if (specialised_off()) return false;
    switch (tw->M) {
        case 32: return col_r_go<T, S, 8, 4, 16>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
        case 64: return col_r_go<T, S, 8, 8, 16>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
        case 128: return col_r_go<T, S, 16, 8, 16>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
        case 160: return col_r_go<T, S, 10, 16, 16>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
        case 270: return col_r_go<T, S, 15, 18, 16>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
        case 512:  // 16 x 32 (32-point register DFTs); 8 columns per block in FP64 (registers)
            if constexpr (sizeof(T) == 4)
                return col_r_go<T, S, 16, 32, 16>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
            else
                return col_r_go<T, S, 16, 32, 8>(in, out, tw, H, Lin, Lout, planes, ips, ops, st, nptr, ell, slot_stride);
        default: return false;
    }
}

template <class Src, typename T>
mot_status launch_xy_forward(Src x, cplx<T> *out, int planes, int Nx, int Ny, int H, AxisTw *tx, AxisTw *ty,
                             cudaStream_t st) {
    if (xy_forward_r<Src, T>(x, out, planes, Nx, Ny, tx, ty, st)) {
        MOT_CHECK_LAUNCH();
        return MOT_OK;
    }
    size_t smem = xy_smem_bytes<T>(tx->M, ty->M, H, Ny);
    MOT_TRY(allow_smem<k_xy_forward<Src, T>>());
    count_launch();
    k_xy_forward<Src, T><<<planes, kXYThreadsOf<T>, smem, st>>>(x, out, Nx, Ny, H, planp<T>(tx), planp<T>(ty), twp<T>(tx), twp<T>(ty));
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

template <typename T, class Epi>
mot_status launch_xy_inverse(const cplx<T> *in, int planes, int Nx, int Ny, int Nz, int H, AxisTw *tx, AxisTw *ty,
                             Epi epi, cudaStream_t st) {
    if (xy_inverse_r<T, Epi>(in, planes, Nx, Ny, Nz, tx, ty, epi, st)) {
        MOT_CHECK_LAUNCH();
        return MOT_OK;
    }
    size_t smem = xy_smem_bytes<T>(tx->M, ty->M, H, Ny);
    MOT_TRY(allow_smem<k_xy_inverse<T, Epi>>());
    count_launch();
    k_xy_inverse<T, Epi><<<planes, kXYThreadsOf<T>, smem, st>>>(in, Nx, Ny, Nz, H, planp<T>(tx), planp<T>(ty), twp<T>(tx), twp<T>(ty), epi);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

template <typename T> const T *L0_of(mot_problem *p);

// specialised z pass when M0z = R1 * R2 is one of the compiled shapes;
// returns false to fall back to the generic pass
// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
using TmapEncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
TmapEncodeFn tmap_encoder() {
    static TmapEncodeFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<TmapEncodeFn>(f);
    }();
    return fn;
}

// the z pass's descriptor over the planes buffer [rows = nrhs 3 Nz][ncols] of
// complex T, viewed as rows of 2 ncols scalars; box 2 TC scalars x Nz rows.
// nullptr where TMA cannot address it (row pitch off the 16-byte grid, box too tall)
template <typename T> const CUtensorMap *z_tmap(mot_problem *p, const cplx<T> *buf, long rows, long ncols, int Nz, int TC) {
    for (auto &z : p->zmaps)
        if (z.ptr == buf && z.rows == rows && z.ncols == ncols && z.Nz == Nz && z.TC == TC && z.es == (int)sizeof(T))
            return &z.map;
    TmapEncodeFn enc = tmap_encoder();
    if (!enc || Nz > 256 || (ncols * (long)sizeof(cplx<T>)) % 16 != 0 || ((uintptr_t)buf & 15) != 0) return nullptr;
    mot_problem::ZMap z;
    z.ptr = buf;
    z.rows = rows;
    z.ncols = ncols;
    z.Nz = Nz;
    z.TC = TC;
    z.es = (int)sizeof(T);
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * ncols), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ncols * sizeof(cplx<T>))};
    const cuuint32_t box[2] = {(cuuint32_t)(2 * TC), (cuuint32_t)Nz};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(&z.map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                           (void *)buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return nullptr;
    p->zmaps.push_back(z);
    return &p->zmaps.back().map;
}

inline bool z_tma_wanted() {
    static const int f = getenv("MOTJVIE_Z_TMA") ? atoi(getenv("MOTJVIE_Z_TMA")) : -1;
    return f >= 0 ? f != 0 : cur_sched().z_tma != 0;
}

template <typename T, int R1, int R2, int TC>
bool z_green_r_tc(mot_problem *p, cplx<T> *Bf, AxisTw *tz, int nrhs, cudaStream_t st) {
    const int My = p->M0[1], H = p->H0, Nz = p->N[2];
    constexpr size_t smem = z_green_r_smem<T, R1, R2, TC>();
    if (smem > kSmemMax || allow_smem<k_z_green_r<T, R1, R2, TC>>() != MOT_OK) return false;
    Octant oc = {p->M0[2], My, p->K0[2], p->K0[1], H};
    dim3 grid((My * H + TC - 1) / TC, (unsigned)nrhs);
    constexpr size_t smem_t = z_green_r_smem_tma<T, R1, R2, TC>();
    const CUtensorMap *tm = nullptr;
    if (z_tma_wanted() && smem_t <= kSmemMax && allow_smem<k_z_green_r<T, R1, R2, TC, true>>() == MOT_OK)
        tm = z_tmap<T>(p, Bf, (long)nrhs * 3 * Nz, (long)My * H, Nz, TC);
    if (!p->capturing) p->kt.begin(st, MOT_K_Z_GREEN);
    count_launch();
    if (tm)
        launch_chain(k_z_green_r<T, R1, R2, TC, true>, grid, dim3(3 * TC * R2), smem_t, st, Bf, L0_of<T>(p),
                     twp<T>(tz), Nz, My, H, oc, *tm);
    else {
        CUtensorMap none;
        memset(&none, 0, sizeof none);
        launch_chain(k_z_green_r<T, R1, R2, TC, false>, grid, dim3(3 * TC * R2), smem, st, Bf, L0_of<T>(p),
                     twp<T>(tz), Nz, My, H, oc, none);
    }
    if (!p->capturing) p->kt.end(st);
    return true;
}

// columns per block TC: 8 (measured fastest for one and for sixteen
// right-hand sides on the 72^3 grid), 16 or 32 where that block would not
// fit; MOTJVIE_Z_COLS = 4 | 8 | 16 | 32 forces one for timing sweeps
template <typename T, int R1, int R2, int TC> constexpr bool z_tc_ok() {
    return 3 * TC * R2 <= 1024 && z_green_r_smem<T, R1, R2, TC>() <= kSmemMax;
}

inline int z_cols_forced() {
    static const int f = getenv("MOTJVIE_Z_COLS") ? atoi(getenv("MOTJVIE_Z_COLS")) : 0;
    return f ? f : cur_sched().z_cols;
}

template <typename T, int R1, int R2> bool z_green_r_go(mot_problem *p, cplx<T> *Bf, AxisTw *tz, int nrhs, cudaStream_t st) {
    const int f = z_cols_forced();
    if constexpr (z_tc_ok<T, R1, R2, 4>())
        if (f == 4) return z_green_r_tc<T, R1, R2, 4>(p, Bf, tz, nrhs, st);
    if constexpr (z_tc_ok<T, R1, R2, 32>())
        if (f == 32) return z_green_r_tc<T, R1, R2, 32>(p, Bf, tz, nrhs, st);
    if constexpr (z_tc_ok<T, R1, R2, 16>())
        if (f == 16) return z_green_r_tc<T, R1, R2, 16>(p, Bf, tz, nrhs, st);
    if constexpr (z_tc_ok<T, R1, R2, 8>()) return z_green_r_tc<T, R1, R2, 8>(p, Bf, tz, nrhs, st);
    else if constexpr (z_tc_ok<T, R1, R2, 16>()) return z_green_r_tc<T, R1, R2, 16>(p, Bf, tz, nrhs, st);
    else return false;
}

template <typename T> bool launch_z_green_r(mot_problem *p, cplx<T> *Bf, AxisTw *tz, int nrhs, cudaStream_t st) {
    if (specialised_off()) return false;
    switch (p->M0[2]) {
        case 20: return z_green_r_go<T, 5, 4>(p, Bf, tz, nrhs, st);
        case 32: return z_green_r_go<T, 8, 4>(p, Bf, tz, nrhs, st);
        case 64: return z_green_r_go<T, 8, 8>(p, Bf, tz, nrhs, st);
        case 72: return z_green_r_go<T, 9, 8>(p, Bf, tz, nrhs, st);
        case 75: return z_green_r_go<T, 5, 15>(p, Bf, tz, nrhs, st);
        case 80: return z_green_r_go<T, 5, 16>(p, Bf, tz, nrhs, st);
        case 90: return z_green_r_go<T, 9, 10>(p, Bf, tz, nrhs, st);
        case 128: return z_green_r_go<T, 16, 8>(p, Bf, tz, nrhs, st);
        default: return false;
    }
}

template <typename T> const T *eps_of(mot_problem *p);
template <> const double *eps_of<double>(mot_problem *p) { return (const double *)p->eps.p; }
template <> const float *eps_of<float>(mot_problem *p) { return (const float *)p->eps32.p; }

template <typename T> const T *L0_of(mot_problem *p);
template <> const double *L0_of<double>(mot_problem *p) { return (const double *)p->L0_64.p; }
template <> const float *L0_of<float>(mot_problem *p) { return (const float *)p->L0_32.p; }
template <> const dfl *L0_of<dfl>(mot_problem *p) { return (const dfl *)p->L0_df.p; }
template <typename T> const T *Lh_of(mot_problem *p);
template <> const double *Lh_of<double>(mot_problem *p) { return (const double *)p->Lh_64.p; }
template <> const float *Lh_of<float>(mot_problem *p) { return (const float *)p->Lh_32.p; }
template <> const dfl *Lh_of<dfl>(mot_problem *p) { return (const dfl *)p->Lh_df.p; }

// timing-option class of a forward source / inverse epilogue
template <class S> struct FwdClass { static constexpr int v = MOT_K_FWD_PLAIN; };
template <typename V> struct FwdClass<SrcHalfA<V>> { static constexpr int v = MOT_K_FWD_HALF; };
template <typename V> struct FwdClass<SrcY1<V>> { static constexpr int v = MOT_K_FWD_Y1; };
template <class E> struct InvClass { static constexpr int v = MOT_K_INV_Z0; };
template <typename V> struct InvClass<EpiHalfB<V>> { static constexpr int v = MOT_K_INV_HALF; };
template <typename V> struct InvClass<EpiV<V>> { static constexpr int v = MOT_K_INV_V; };
template <> struct InvClass<EpiResidual> { static constexpr int v = MOT_K_INV_RESIDUAL; };

// true if the present-time xy passes run as one plane per block
template <typename T> bool z0_planes_fit(const mot_problem *p) {
    return xy_smem_bytes<T>(p->M0[0], p->M0[1], p->H0, p->N[1]) <= kSmemMax;
}

// y = Z0 x (or the residual epilogue) with the FFT in precision T.  The
// input comes from src (a stored vector or one formed on the fly); the row
// passes used when a plane does not fit in shared memory read `plain`, which
// must then hold the same vector (nullptr: that case is refused).
// wsA: nrhs*3*Nz*Ny*H0 complex, wsB: nrhs*3*Nz*M0y*H0 complex.
template <class Src, typename TI, typename T, class Epi>
mot_status z0_product_src(mot_problem *p, Src src, const TI *plain, int nrhs, void *wsA, void *wsB, Epi epi,
                          cudaStream_t st) {
    const int Nx = p->N[0], Ny = p->N[1], Nz = p->N[2];
    const int H = p->H0, My = p->M0[1];
    AxisTw *tx = get_tw(p, p->M0[0]), *ty = get_tw(p, p->M0[1]), *tz = get_tw(p, p->M0[2]);
    if (!tx || !ty || !tz) MOT_FAIL(MOT_EUNSUPPORTED, "FFT size with a prime factor above 5");
    using C = cplx<T>;
    C *A = (C *)wsA, *Bf = (C *)wsB;
    const long nrows = (long)nrhs * 3 * Nz * Ny;
    const int planes = nrhs * 3 * Nz;
    const bool fused = z0_planes_fit<T>(p);
    const bool timed = !p->capturing;
    if (fused) {
        if (timed) p->kt.begin(st, FwdClass<Src>::v);
        MOT_TRY((launch_xy_forward<Src, T>(src, Bf, planes, Nx, Ny, H, tx, ty, st)));
        if (timed) p->kt.end(st);
    }
    else if constexpr (Epi::kPlaneOnly) {
        MOT_FAIL(MOT_EUNSUPPORTED, "fused solver epilogue needs the plane passes");
    } else {
        if (!plain) MOT_FAIL(MOT_EUNSUPPORTED, "row-pass product needs a stored input vector");
        if (timed) p->kt.begin(st, MOT_K_ROW_FWD);
        if (x_forward_r<TI, T>(plain, A, nrows, Nx, Ny, tx, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY(launch_x_forward<TI, T>(plain, A, nrows, Nx, H, tx, st));
        if (col_r<T, -1>(A, Bf, ty, H, Ny, My, planes, (long)Ny * H, (long)My * H, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_axis<T, -1>(A, Bf, ty, H, Ny, My, planes, 1, (long)Ny * H, 0, H, (long)My * H, 0, H, st)));
        if (timed) p->kt.end(st);
    }
    if (launch_z_green_r<T>(p, Bf, tz, nrhs, st)) {
        MOT_CHECK_LAUNCH();
    } else {
        int tw = tile_width<T>(p->M0[2], 3);
        size_t smem = (size_t)(6 * p->M0[2] * tw + p->M0[2]) * sizeof(C);
        MOT_TRY(allow_smem<k_z_green<T>>());
        Octant oc = {p->M0[2], p->M0[1], p->K0[2], p->K0[1], H};
        dim3 grid((H + tw - 1) / tw, (unsigned)(nrhs * My));
        if (!p->capturing) p->kt.begin(st, MOT_K_Z_GREEN);
        count_launch();
        k_z_green<T><<<grid, kZThreads, smem, st>>>(Bf, L0_of<T>(p), planp<T>(tz), twp<T>(tz), Nz, My, H, tw, oc);
        if (!p->capturing) p->kt.end(st);
        MOT_CHECK_LAUNCH();
    }
    if (fused) {
        if (timed) p->kt.begin(st, InvClass<Epi>::v);
        MOT_TRY(launch_xy_inverse<T, Epi>(Bf, planes, Nx, Ny, Nz, H, tx, ty, epi, st));
        if (timed) p->kt.end(st);
    } else if constexpr (!Epi::kPlaneOnly) {
        if (timed) p->kt.begin(st, MOT_K_ROW_INV);
        if (col_r<T, +1>(Bf, A, ty, H, My, Ny, planes, (long)My * H, (long)Ny * H, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_axis<T, +1>(Bf, A, ty, H, My, Ny, planes, 1, (long)My * H, 0, H, (long)Ny * H, 0, H, st)));
        if (x_inverse_r<T, Epi>(A, nrows, Nx, Ny, Nz, tx, epi, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_x_inverse<T, Epi>(A, nrows, Nx, H, tx, epi, st)));
        if (timed) p->kt.end(st);
    }
    return MOT_OK;
}

template <typename TI, typename T, class Epi>
mot_status z0_product(mot_problem *p, const TI *x, int nrhs, void *wsA, void *wsB, Epi epi, cudaStream_t st) {
    return z0_product_src<SrcPlain<TI>, TI, T, Epi>(p, SrcPlain<TI>{x}, x, nrhs, wsA, wsB, epi, st);
}

size_t z0_ws_bytes(const mot_problem *p, int nrhs, size_t csize, size_t *a, size_t *b) {
    *a = (size_t)nrhs * 3 * p->N[2] * p->N[1] * p->H0 * csize;
    *b = (size_t)nrhs * 3 * p->N[2] * p->M0[1] * p->H0 * csize;
    return *a + *b;
}

// ---------------------------------------------------------------- autotuner
// Picks the launch schedule (Sched) of the Z0 product for one (grid, number of
// right-hand sides, precision) by timing candidates with CUDA events on the
// context's stream: coordinate descent over z-pass columns per block, row-pass
// rows per block, plane-pass block sizes, generic-pass row pairs and tile
// widths and programmatic dependent launch, each candidate's product checked
// against the built-in schedule's product (every candidate must give the same
// result; one that does not is discarded and counted).  Results are cached
// per process by (grid, M0, right-hand sides, precision).
template <typename T>
__global__ void k_diff2(const T *__restrict__ a, const T *__restrict__ b, long n, double *__restrict__ acc) {
    double d2 = 0.0, r2 = 0.0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double x = (double)a[i], y = (double)b[i];
        d2 += (x - y) * (x - y);
        r2 += y * y;
    }
    d2 = warp_sum(d2);
    r2 = warp_sum(r2);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, d2);
        atomicAdd(acc + 1, r2);
    }
}

struct TuneCacheEntry {
    int N[3], M0[3], nrhs, fp32;
    Sched s;
    mot_schedule info;
};
std::mutex g_tune_mu;
std::vector<TuneCacheEntry> g_tune_cache;

template <typename T> bool z_cols_valid(int M0z, int tc) {
    auto ok = [&](auto r1, auto r2) {
        constexpr int R1 = decltype(r1)::value, R2 = decltype(r2)::value;
        switch (tc) {
            case 4: return z_tc_ok<T, R1, R2, 4>();
            case 8: return z_tc_ok<T, R1, R2, 8>();
            case 16: return z_tc_ok<T, R1, R2, 16>();
            case 32: return z_tc_ok<T, R1, R2, 32>();
            default: return false;
        }
    };
    using std::integral_constant;
    switch (M0z) {
        case 20: return ok(integral_constant<int, 5>{}, integral_constant<int, 4>{});
        case 32: return ok(integral_constant<int, 8>{}, integral_constant<int, 4>{});
        case 64: return ok(integral_constant<int, 8>{}, integral_constant<int, 8>{});
        case 72: return ok(integral_constant<int, 9>{}, integral_constant<int, 8>{});
        case 75: return ok(integral_constant<int, 5>{}, integral_constant<int, 15>{});
        case 80: return ok(integral_constant<int, 5>{}, integral_constant<int, 16>{});
        case 90: return ok(integral_constant<int, 9>{}, integral_constant<int, 10>{});
        case 128: return ok(integral_constant<int, 16>{}, integral_constant<int, 8>{});
        default: return false;
    }
}

inline bool compiled_plane(int Mx, int My) {
    return Mx == My && (Mx == 20 || Mx == 32 || Mx == 72 || Mx == 75 || Mx == 128);
}
inline bool compiled_col(int M) { return M == 32 || M == 64 || M == 128 || M == 160 || M == 270 || M == 512; }

template <typename T>
mot_status tune_product(mot_problem *p, int nrhs, Sched &best, mot_schedule &info) {
    const bool fp32 = sizeof(T) == 4;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &e : g_tune_cache)
            if (e.nrhs == nrhs && e.fp32 == (int)fp32 && !memcmp(e.N, p->N, sizeof e.N) && !memcmp(e.M0, p->M0, sizeof e.M0)) {
                best = e.s;
                info = e.info;
                info.cached = 1;
                return MOT_OK;
            }
    }
    cudaStream_t st = p->ctx->stream;
    const long n = (long)nrhs * 3 * p->N[0] * p->N[1] * p->N[2];
    size_t a, b;
    z0_ws_bytes(p, nrhs, sizeof(cplx<T>), &a, &b);
    DBuf x, y, yref, wa, wb, acc;
    MOT_TRY(dalloc(x, sizeof(T) * n));
    MOT_TRY(dalloc(y, sizeof(T) * n));
    MOT_TRY(dalloc(yref, sizeof(T) * n));
    MOT_TRY(dalloc(wa, a));
    MOT_TRY(dalloc(wb, b));
    MOT_TRY(dalloc(acc, 2 * sizeof(double)));
    {   // a fixed pseudo-random input (any input gives the same timing)
        std::vector<T> hx(n);
        uint64_t z = 0x9E3779B97F4A7C15ull;
        for (long i = 0; i < n; ++i) {
            z ^= z << 13;
            z ^= z >> 7;
            z ^= z << 17;
            hx[i] = (T)((double)(z >> 11) * 0x1.0p-53 - 0.5);
        }
        MOT_CUDA_TRY(cudaMemcpyAsync(x.p, hx.data(), sizeof(T) * n, cudaMemcpyHostToDevice, st));
        MOT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    const long pr = (long)p->N[2] * p->N[1];
    cudaEvent_t e0, e1;
    MOT_CUDA_TRY(cudaEventCreate(&e0));
    MOT_CUDA_TRY(cudaEventCreate(&e1));
    const bool was = p->capturing;
    p->capturing = true;  // no kernel-timing events while tuning
    auto run = [&](const Sched &s, T *out) -> mot_status {
        SchedScope sc(&s);
        EpiZ0<T, T> e = {(const T *)x.p, out, eps_of<T>(p), pr, p->N[0], (T)p->opt.delta};
        return z0_product<T, T>(p, (const T *)x.p, nrhs, wa.p, wb.p, e, st);
    };
    int reps = 3;
    auto timeit = [&](const Sched &s, float *ms) -> mot_status {
        for (int w = 0; w < 2; ++w) MOT_TRY(run(s, (T *)y.p));
        float bestb = 1e30f;
        for (int batch = 0; batch < 3; ++batch) {
            MOT_CUDA_TRY(cudaEventRecord(e0, st));
            for (int r = 0; r < reps; ++r) MOT_TRY(run(s, (T *)y.p));
            MOT_CUDA_TRY(cudaEventRecord(e1, st));
            MOT_CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            MOT_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            bestb = std::min(bestb, t / reps);
        }
        *ms = bestb;
        return MOT_OK;
    };
    auto diff = [&](double *rel) -> mot_status {
        MOT_CUDA_TRY(cudaMemsetAsync(acc.p, 0, 2 * sizeof(double), st));
        count_launch();
        k_diff2<T><<<grid_for(n), 256, 0, st>>>((const T *)y.p, (const T *)yref.p, n, (double *)acc.p);
        MOT_CHECK_LAUNCH();
        double h[2];
        MOT_CUDA_TRY(cudaMemcpyAsync(h, acc.p, sizeof h, cudaMemcpyDeviceToHost, st));
        MOT_CUDA_TRY(cudaStreamSynchronize(st));
        *rel = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
        return MOT_OK;
    };
    mot_status rc = MOT_OK;
    memset(&info, 0, sizeof info);
    do {
        Sched base;
        if ((rc = run(base, (T *)yref.p)) != MOT_OK) break;
        float t1 = 0.f;
        MOT_CUDA_TRY(cudaEventRecord(e0, st));
        if ((rc = run(base, (T *)y.p)) != MOT_OK) break;
        MOT_CUDA_TRY(cudaEventRecord(e1, st));
        MOT_CUDA_TRY(cudaEventSynchronize(e1));
        MOT_CUDA_TRY(cudaEventElapsedTime(&t1, e0, e1));
        reps = std::max(3, std::min(30, (int)ceil(2.0 / std::max(1e-3f, t1))));
        float tbest = 0.f;
        if ((rc = timeit(base, &tbest)) != MOT_OK) break;
        info.ms_default = tbest;
        best = base;
        // candidate values per dimension, for the passes this product uses
        const bool fused = z0_planes_fit<T>(p);
        const bool zc = z_cols_valid<T>(p->M0[2], 8) || z_cols_valid<T>(p->M0[2], 16);
        const bool rows270 = !fused && p->M0[0] == 270;
        const bool gen_x = !fused ? p->M0[0] != 270 : !compiled_plane(p->M0[0], p->M0[1]);
        const bool gen_axis = fused ? !compiled_plane(p->M0[0], p->M0[1]) : !compiled_col(p->M0[1]);
        struct Dim {
            int Sched::*f;
            std::vector<int> v;
        };
        std::vector<Dim> dims;
        if (zc) {
            std::vector<int> v;
            for (int c : {4, 8, 16, 32})
                if (z_cols_valid<T>(p->M0[2], c)) v.push_back(c);
            dims.push_back({&Sched::z_cols, v});
            dims.push_back({&Sched::z_tma, {1}});
        }
        if (rows270) {
            std::vector<int> v;
            for (int r : {8, 16, 32})
                if (p->N[1] % r == 0) v.push_back(r);
            dims.push_back({&Sched::x_rows, v});
        }
        if (fused && compiled_plane(p->M0[0], p->M0[1]) && fp32) {
            dims.push_back({&Sched::xy_fwd, {256, 384, 512}});
            dims.push_back({&Sched::xy_inv, {256, 384, 512}});
        }
        if (gen_x) dims.push_back({&Sched::gen_pairs, {1, 2, 4, 8}});
        if (gen_axis) dims.push_back({&Sched::gen_tile, {1, 2, 4, 8, 16}});
        dims.push_back({&Sched::pdl, {1, 0}});
        for (auto &d : dims) {
            for (int v : d.v) {
                Sched c = best;
                c.*(d.f) = v;
                float t = 0.f;
                if ((rc = timeit(c, &t)) != MOT_OK) break;
                double rel = 0.0;
                if ((rc = diff(&rel)) != MOT_OK) break;
                info.candidates += 1;
                info.max_rel_diff = std::max(info.max_rel_diff, rel);
                if (rel > (fp32 ? 1e-6 : 1e-13)) {
                    info.rejected += 1;
                    continue;
                }
                if (t < 0.99f * tbest) {
                    tbest = t;
                    best = c;
                }
            }
            if (rc != MOT_OK) break;
        }
        if (rc != MOT_OK) break;
        info.ms_tuned = tbest;
    } while (0);
    p->capturing = was;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MOT_OK) return rc;
    info.z_cols = best.z_cols;
    info.x_rows = best.x_rows;
    info.xy_fwd = best.xy_fwd;
    info.xy_inv = best.xy_inv;
    info.pdl = best.pdl;
    info.gen_pairs = best.gen_pairs;
    info.gen_tile = best.gen_tile;
    info.z_tma = best.z_tma;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        TuneCacheEntry e;
        memcpy(e.N, p->N, sizeof e.N);
        memcpy(e.M0, p->M0, sizeof e.M0);
        e.nrhs = nrhs;
        e.fp32 = fp32;
        e.s = best;
        e.info = info;
        g_tune_cache.push_back(e);
    }
    return MOT_OK;
}

// the problem's schedule for (nrhs, precision), tuned on first use when the
// problem's options ask for it (nullptr: built-in rules)
template <typename T> mot_status schedule_for(mot_problem *p, int nrhs, const Sched **out) {
    const bool fp32 = sizeof(T) == 4;
    *out = p->sched_for(nrhs, fp32);
    if (*out || !p->opt.autotune) return MOT_OK;
    mot_problem::Tuned t;
    t.nrhs = nrhs;
    t.fp32 = fp32;
    MOT_TRY(tune_product<T>(p, nrhs, t.s, t.info));
    p->tuned.push_back(t);
    *out = p->sched_for(nrhs, fp32);
    return MOT_OK;
}

// ---------------------------------------------------------------- tables
// octant of lag k from the library's own quadrature (device), into lags[k]
mot_status compute_lag_octants(mot_problem *p, int k0, int k1) {
    cudaStream_t st = p->ctx->stream;
    int ext[3];
    for (int i = 0; i < 3; ++i) ext[i] = p->N[i] - 1;
    int S[3] = {ext[0], ext[1], ext[2]};
    std::sort(S, S + 3);
    int rmax = lag_reach(k1, p->rho);
    for (int i = 0; i < 3; ++i) S[i] = std::min(S[i], rmax);
    ItemSet is;
    PhaseTrace tr_all("lag tables (items, quadrature or cache, octants)");
    // a cached quadrature brings the item ranges with it: the host item set is built on a miss only
    auto hit = tcache_find(p->rho, S, k0, k1);
    if (!hit) {
        PhaseTrace tr_items("lag-table items (host)");
        if (!build_items(p->rho, S, k0, k1, is))
            MOT_FAIL(MOT_EUNSUPPORTED, "time step too small for the lag-table quadrature (alpha < 0.5)");
    }
    const int nit = hit ? (int)(hit->A6.size() / 6) : (int)is.items.size();
    const int Rm = hit ? hit->Rm : is.Rm;
    const std::vector<int> &rbase = hit ? hit->base : is.base, &rklo = hit ? hit->klo : is.klo,
                           &rcnt = hit ? hit->cnt : is.cnt;
    DBuf dA, dmap;
    MOT_TRY(dalloc(dA, sizeof(double) * 6 * std::max(1, nit)));
    MOT_TRY(dalloc(dmap, sizeof(int) * rbase.size()));
    if (hit && nit > 0) {
        MOT_CUDA_TRY(cudaMemcpyAsync(dA.p, hit->A6.data(), sizeof(double) * 6 * nit, cudaMemcpyHostToDevice, st));
        MOT_CUDA_TRY(cudaStreamSynchronize(st));
    } else if (nit > 0) {
        const int nf = (int)is.faces.size(), nt = (int)is.tri.size();
        DBuf ditems, dfaces, dtri, dFM, dBM;
        MOT_TRY(dalloc(ditems, sizeof(TableItem) * nit));
        MOT_TRY(dalloc(dfaces, sizeof(FaceRec) * std::max(1, nf)));
        MOT_TRY(dalloc(dtri, sizeof(TripleRec) * std::max(1, nt)));
        MOT_TRY(dalloc(dFM, sizeof(double) * std::max(1L, is.fm_len)));
        MOT_TRY(dalloc(dBM, sizeof(double) * std::max(1L, is.bm_len)));
        MOT_CUDA_TRY(cudaMemcpyAsync(ditems.p, is.items.data(), sizeof(TableItem) * nit, cudaMemcpyHostToDevice, st));
        MOT_CUDA_TRY(cudaMemcpyAsync(dfaces.p, is.faces.data(), sizeof(FaceRec) * nf, cudaMemcpyHostToDevice, st));
        MOT_CUDA_TRY(cudaMemcpyAsync(dtri.p, is.tri.data(), sizeof(TripleRec) * nt, cudaMemcpyHostToDevice, st));
        const double *glx = (const double *)p->glx.p, *glw = (const double *)p->glw.p;
        count_launch();
        k_face_moments<<<(nf + 63) / 64, 64, 0, st>>>((const FaceRec *)dfaces.p, nf, p->rho, glx, glw, kGLN,
                                                      (double *)dFM.p);
        MOT_CHECK_LAUNCH();
        count_launch();
        k_box_moments<<<(nt + 63) / 64, 64, 0, st>>>((const TripleRec *)dtri.p, nt, p->rho, glx, glw, kGLN, kGL8,
                                                     (double *)dBM.p);
        MOT_CHECK_LAUNCH();
        count_launch();
        k_combine_items<<<(nit + 255) / 256, 256, 0, st>>>((const TableItem *)ditems.p, nit,
                                                           (const TripleRec *)dtri.p, (const FaceRec *)dfaces.p,
                                                           (const double *)dFM.p, (const double *)dBM.p,
                                                           (double *)dA.p);
        MOT_CHECK_LAUNCH();
        std::vector<double> A6(6 * (size_t)nit);
        MOT_CUDA_TRY(cudaMemcpyAsync(A6.data(), dA.p, sizeof(double) * 6 * nit, cudaMemcpyDeviceToHost, st));
        MOT_CUDA_TRY(cudaStreamSynchronize(st));
        tcache_put(p->rho, S, k0, k1, std::move(A6), is);
        dfree(ditems);
        dfree(dfaces);
        dfree(dtri);
        dfree(dFM);
        dfree(dBM);
    }
    // each lag's item map is formed on the device from the per-offset item ranges
    const long n3 = (long)rbase.size();
    DBuf drange;
    MOT_TRY(dalloc(drange, sizeof(int) * 3 * n3));
    int *dbase = (int *)drange.p, *dklo = dbase + n3, *dcnt = dklo + n3;
    MOT_CUDA_TRY(cudaMemcpyAsync(dbase, rbase.data(), sizeof(int) * n3, cudaMemcpyHostToDevice, st));
    MOT_CUDA_TRY(cudaMemcpyAsync(dklo, rklo.data(), sizeof(int) * n3, cudaMemcpyHostToDevice, st));
    MOT_CUDA_TRY(cudaMemcpyAsync(dcnt, rcnt.data(), sizeof(int) * n3, cudaMemcpyHostToDevice, st));
    for (int k = k0; k <= k1; ++k) {
        LagTable &L = p->lags[k];
        if (L.override_) continue;
        int rk = lag_reach(k, p->rho);
        for (int i = 0; i < 3; ++i) L.R[i] = std::min(rk, ext[i]);
        long n = (long)(L.R[0] + 1) * (L.R[1] + 1) * (L.R[2] + 1);
        MOT_TRY(dalloc(L.oct, sizeof(double) * 6 * n));
        count_launch();
        k_lag_map<<<grid_for(n3), 256, 0, st>>>(dbase, dklo, dcnt, n3, k, (int *)dmap.p);
        count_launch();
        k_expand_octant<<<grid_for(n), 256, 0, st>>>((const double *)dA.p, (const int *)dmap.p, Rm, L.R[0],
                                                     L.R[1], L.R[2], (double *)L.oct.p);
        MOT_CHECK_LAUNCH();
        L.ready = true;
    }
    MOT_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(dA);
    dfree(dmap);
    dfree(drange);
    return MOT_OK;
}

// Lambda of one lag octant on grid M (K = M/2+1), FP64, into dst64 [6][Kz][Ky][Kx]
// Lambda of one lag table: three separable passes over the octant (section on
// tables.cuh).  df: the passes as double-float matrix products (k_gemm_df,
// relative error about 1e-14, several times the FP64 rate of this GPU); else
// plain FP64 sums.  The history lags take df, Lambda0 (the product's own
// spectrum) FP64; MOTJVIE_SPECTRA_FP64=1 keeps every lag in FP64.
mot_status lag_spectrum(mot_problem *p, const LagTable &L, const int M[3], double *dst64, bool df = false) {
    static const bool force64 = getenv("MOTJVIE_SPECTRA_FP64") && atoi(getenv("MOTJVIE_SPECTRA_FP64")) != 0;
    if (force64) df = false;
    cudaStream_t st = p->ctx->stream;
    int K[3] = {M[0] / 2 + 1, M[1] / 2 + 1, M[2] / 2 + 1};
    int R1[3] = {L.R[0] + 1, L.R[1] + 1, L.R[2] + 1};
    std::vector<double> ce[3], co[3];
    for (int a = 0; a < 3; ++a) {
        axis_coef(M[a], L.R[a], false, ce[a]);
        axis_coef(M[a], L.R[a], true, co[a]);
    }
    DBuf dce[3], dco[3], t1, t2;
    for (int a = 0; a < 3; ++a) {
        MOT_TRY(dalloc(dce[a], sizeof(double) * ce[a].size()));
        MOT_TRY(dalloc(dco[a], sizeof(double) * co[a].size()));
        MOT_CUDA_TRY(cudaMemcpyAsync(dce[a].p, ce[a].data(), sizeof(double) * ce[a].size(), cudaMemcpyHostToDevice, st));
        MOT_CUDA_TRY(cudaMemcpyAsync(dco[a].p, co[a].data(), sizeof(double) * co[a].size(), cudaMemcpyHostToDevice, st));
    }
    MOT_TRY(dalloc(t1, sizeof(double) * (size_t)R1[2] * R1[1] * K[0]));
    MOT_TRY(dalloc(t2, sizeof(double) * (size_t)R1[2] * K[1] * K[0]));
    const long on = (long)R1[0] * R1[1] * R1[2];
    const long kn = (long)K[0] * K[1] * K[2];
    const double scale = 1.0 / ((double)M[0] * M[1] * M[2]);
    // parity per component (x, y, z): 1 = odd
    const int par[6][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int c = 0; c < 6; ++c) {
        const double *src = (const double *)L.oct.p + c * on;
        const double *cx = (const double *)(par[c][0] ? dco[0].p : dce[0].p);
        const double *cy = (const double *)(par[c][1] ? dco[1].p : dce[1].p);
        const double *cz = (const double *)(par[c][2] ? dco[2].p : dce[2].p);
        if (df) {
            const double s = c >= 3 ? -scale : scale;
            const int M1 = R1[2] * R1[1];
            count_launch();
            k_gemm_df<<<dim3((K[0] + 63) / 64, (M1 + 63) / 64, 1), 256, 0, st>>>(
                GemmView{src, 0, R1[0], 1}, GemmView{cx, 0, 1, R1[0]}, (double *)t1.p, 0, K[0], 1, M1, K[0], R1[0], 1.0);
            count_launch();
            k_gemm_df<<<dim3((K[0] + 63) / 64, (K[1] + 63) / 64, R1[2]), 256, 0, st>>>(
                GemmView{cy, 0, R1[1], 1}, GemmView{(const double *)t1.p, (long)R1[1] * K[0], K[0], 1}, (double *)t2.p,
                (long)K[1] * K[0], K[0], 1, K[1], K[0], R1[1], 1.0);
            const int NN = K[1] * K[0];
            count_launch();
            k_gemm_df<<<dim3((NN + 63) / 64, (K[2] + 63) / 64, 1), 256, 0, st>>>(
                GemmView{cz, 0, R1[2], 1}, GemmView{(const double *)t2.p, 0, NN, 1}, dst64 + c * kn, 0, NN, 1, K[2], NN,
                R1[2], s);
            MOT_CHECK_LAUNCH();
            continue;
        }
        long n1 = (long)R1[2] * R1[1] * K[0];
        count_launch();
        k_axis_sum<<<grid_for(n1), 256, 0, st>>>(src, (double *)t1.p, cx, R1[2] * R1[1], R1[0], K[0], 1);
        long n2 = (long)R1[2] * K[1] * K[0];
        count_launch();
        k_axis_sum<<<grid_for(n2), 256, 0, st>>>((const double *)t1.p, (double *)t2.p, cy, R1[2], R1[1], K[1], K[0]);
        count_launch();
        k_axis_sum<<<grid_for(kn), 256, 0, st>>>((const double *)t2.p, dst64 + c * kn, cz, 1, R1[2], K[2],
                                                 K[1] * K[0]);
        MOT_CHECK_LAUNCH();
        double s = c >= 3 ? -scale : scale;
        count_launch();
        k_scale_store<double><<<grid_for(kn), 256, 0, st>>>(dst64 + c * kn, dst64 + c * kn, kn, s);
        MOT_CHECK_LAUNCH();
    }
    MOT_CUDA_TRY(cudaStreamSynchronize(st));
    for (int a = 0; a < 3; ++a) {
        dfree(dce[a]);
        dfree(dco[a]);
    }
    dfree(t1);
    dfree(t2);
    return MOT_OK;
}

mot_status build_Z0_spectrum(mot_problem *p) {
    long kn = (long)p->K0[0] * p->K0[1] * p->K0[2];
    MOT_TRY(dalloc(p->L0_64, sizeof(double) * 6 * kn));
    MOT_TRY(dalloc(p->L0_32, sizeof(float) * 6 * kn));
    MOT_TRY(dalloc(p->L0_df, sizeof(dfl) * 6 * kn));
    MOT_TRY(lag_spectrum(p, p->lags[0], p->M0, (double *)p->L0_64.p));
    count_launch();
    k_scale_store<float><<<grid_for(6 * kn), 256, 0, p->ctx->stream>>>((const double *)p->L0_64.p,
                                                                       (float *)p->L0_32.p, 6 * kn, 1.0);
    MOT_CHECK_LAUNCH();
    count_launch();
    k_scale_store<dfl><<<grid_for(6 * kn), 256, 0, p->ctx->stream>>>((const double *)p->L0_64.p,
                                                                     (dfl *)p->L0_df.p, 6 * kn, 1.0);
    MOT_CHECK_LAUNCH();
    MOT_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
    return MOT_OK;
}

// process-wide registry of history spectra on the device: problems with the
// same device, step (rho), grid, history grid and precision and no caller-
// supplied lag tables share one copy (their spectra do not depend on eps_r)
struct SpecKey {
    int device;
    double rho;
    int N[3], Mh[3], ell, kind;
    bool operator==(const SpecKey &o) const {
        return device == o.device && rho == o.rho && !memcmp(N, o.N, sizeof N) && !memcmp(Mh, o.Mh, sizeof Mh) &&
               ell == o.ell && kind == o.kind;
    }
};
std::mutex g_spec_mu;
std::vector<std::pair<SpecKey, std::weak_ptr<SharedDev>>> g_spec;

SpecKey spec_key(const mot_problem *p, int kind) {
    SpecKey k;
    k.device = p->ctx->device;
    k.rho = p->rho;
    for (int i = 0; i < 3; ++i) {
        k.N[i] = p->N[i];
        k.Mh[i] = p->Mh[i];
    }
    k.ell = p->ell;
    k.kind = kind;
    return k;
}

std::shared_ptr<SharedDev> spec_lookup(const SpecKey &k) {
    std::lock_guard<std::mutex> lk(g_spec_mu);
    for (auto it = g_spec.begin(); it != g_spec.end();) {
        if (it->second.expired()) {
            it = g_spec.erase(it);
            continue;
        }
        if (it->first == k) return it->second.lock();
        ++it;
    }
    return nullptr;
}

// hand the problem's own spectra buffer over to a shared holder and register it
void spec_share(mot_problem *p, DBuf &buf, int kind) {
    auto h = std::make_shared<SharedDev>();
    h->p = buf.p;
    h->bytes = buf.bytes;
    h->device = p->ctx->device;
    p->lh_hold[kind] = h;
    std::lock_guard<std::mutex> lk(g_spec_mu);
    g_spec.emplace_back(spec_key(p, kind), h);
}

// history spectra of one arithmetic: FP64, FP32 or double-float (kinds below),
// computed in FP64 per lag and stored in that arithmetic
enum { kSpec64 = 0, kSpec32 = 1, kSpecDF = 2 };
DBuf &spec_buf(mot_problem *p, int kind) { return kind == kSpec64 ? p->Lh_64 : kind == kSpec32 ? p->Lh_32 : p->Lh_df; }
bool &spec_have(mot_problem *p, int kind) { return kind == kSpec64 ? p->hist64 : kind == kSpec32 ? p->hist32 : p->histdf; }

mot_status build_history_spectra(mot_problem *p, int kind) {
    bool &have = spec_have(p, kind);
    if (have) return MOT_OK;
    DBuf &buf = spec_buf(p, kind);
    bool shareable = true;  // no caller-supplied table among the history lags
    for (int k = 1; k <= p->ell; ++k)
        if (p->lags[k].override_) shareable = false;
    if (shareable) {
        if (auto h = spec_lookup(spec_key(p, kind))) {
            dfree(buf);
            buf.p = h->p;
            buf.bytes = h->bytes;
            p->lh_hold[kind] = h;
            have = true;
            return MOT_OK;
        }
    }
    bool need_oct = false;
    for (int k = 1; k <= p->ell; ++k)
        if (!p->lags[k].ready) need_oct = true;
    if (need_oct) MOT_TRY(compute_lag_octants(p, 1, p->ell));
    PhaseTrace tr_spec("history spectra");
    long kn = (long)p->Kh[0] * p->Kh[1] * p->Kh[2];
    size_t per = 6 * (size_t)kn;
    const size_t es = kind == kSpec32 ? sizeof(float) : sizeof(double);  // a dfl is 8 bytes too
    DBuf tmp;
    if (kind != kSpec64) MOT_TRY(dalloc(tmp, sizeof(double) * per));
    MOT_TRY(dalloc(buf, es * per * (p->ell + 1)));
    MOT_CUDA_TRY(cudaMemsetAsync(buf.p, 0, es * per, p->ctx->stream));
    for (int k = 1; k <= p->ell; ++k) {
        double *dst = kind == kSpec64 ? (double *)buf.p + per * k : (double *)tmp.p;
        MOT_TRY(lag_spectrum(p, p->lags[k], p->Mh, dst, true));
        if (kind == kSpec32) {
            count_launch();
            k_scale_store<float><<<grid_for(per), 256, 0, p->ctx->stream>>>(dst, (float *)buf.p + per * k, per, 1.0);
            MOT_CHECK_LAUNCH();
        } else if (kind == kSpecDF) {
            count_launch();
            k_scale_store<dfl><<<grid_for(per), 256, 0, p->ctx->stream>>>(dst, (dfl *)buf.p + per * k, per, 1.0);
            MOT_CHECK_LAUNCH();
        }
    }
    MOT_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
    dfree(tmp);
    have = true;
    if (shareable) spec_share(p, buf, kind);
    return MOT_OK;
}

// host: octant -> full table with reflection signs
void octant_to_full(const std::vector<double> &oct, const int R[3], double *g) {
    int nx = 2 * R[0] + 1, ny = 2 * R[1] + 1, nz = 2 * R[2] + 1;
    long n3 = (long)nx * ny * nz;
    long on = (long)(R[0] + 1) * (R[1] + 1) * (R[2] + 1);
    const int pp[6] = {0, 1, 2, 0, 0, 1}, qq[6] = {0, 1, 2, 1, 2, 2};
    for (int dz = -R[2]; dz <= R[2]; ++dz)
        for (int dy = -R[1]; dy <= R[1]; ++dy)
            for (int dx = -R[0]; dx <= R[0]; ++dx) {
                int d[3] = {dx, dy, dz};
                long oi = ((long)abs(dz) * (R[1] + 1) + abs(dy)) * (R[0] + 1) + abs(dx);
                long fi = ((long)(dz + R[2]) * ny + (dy + R[1])) * nx + (dx + R[0]);
                for (int c = 0; c < 6; ++c) {
                    double s = 1.0;
                    if (c >= 3) s = (d[pp[c]] < 0 ? -1.0 : 1.0) * (d[qq[c]] < 0 ? -1.0 : 1.0);
                    g[c * n3 + fi] = s * oct[c * on + oi];
                }
            }
}

bool finite_all(const double *a, long n) {
    for (long i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
namespace {
// tile of the direct product: the largest of 8x8x8 .. 4x4x2 whose haloed
// three-component input fits in shared memory
bool direct_tile(const mot_problem *p, size_t es, int *t) {
    const int R[3] = {p->lags[0].R[0], p->lags[0].R[1], p->lags[0].R[2]};
    const int cand[][3] = {{8, 8, 8}, {8, 8, 4}, {8, 4, 4}, {4, 4, 4}, {4, 4, 2}, {4, 2, 2}, {2, 2, 2}};
    for (auto &c : cand) {
        const size_t smem = 3 * es * (size_t)(c[0] + 2 * R[0]) * (c[1] + 2 * R[1]) * (c[2] + 2 * R[2]);
        if (smem <= kSmemMax) {
            t[0] = c[0];
            t[1] = c[1];
            t[2] = c[2];
            return true;
        }
    }
    return false;
}

// the nonzero offsets of the lag-0 table with their signed values, as the
// direct kernel reads them (tile offsets for the haloed tile SX x SY)
template <typename T> mot_status direct_list(mot_problem *p, int SX, int SY) {
    auto &D = p->direct;
    const int fp32 = sizeof(T) == 4;
    if (D.fp32 == fp32 && D.SX == SX && D.SY == SY) return MOT_OK;
    const LagTable &L = p->lags[0];
    const int R[3] = {L.R[0], L.R[1], L.R[2]};
    const long on = (long)(R[0] + 1) * (R[1] + 1) * (R[2] + 1);
    std::vector<double> oct(6 * on);
    MOT_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
    MOT_CUDA_TRY(cudaMemcpy(oct.data(), L.oct.p, sizeof(double) * 6 * on, cudaMemcpyDeviceToHost));
    std::vector<int4> dl;
    std::vector<T> gv;
    for (int dz = -R[2]; dz <= R[2]; ++dz)
        for (int dy = -R[1]; dy <= R[1]; ++dy)
            for (int dx = -R[0]; dx <= R[0]; ++dx) {
                const long oi = ((long)std::abs(dz) * (R[1] + 1) + std::abs(dy)) * (R[0] + 1) + std::abs(dx);
                const double sx = dx < 0 ? -1.0 : 1.0, sy = dy < 0 ? -1.0 : 1.0, sz = dz < 0 ? -1.0 : 1.0;
                double g[6] = {oct[oi], oct[on + oi], oct[2 * on + oi], sx * sy * oct[3 * on + oi],
                               sx * sz * oct[4 * on + oi], sy * sz * oct[5 * on + oi]};
                bool any = false;
                for (double v : g) any = any || v != 0.0;
                if (!any) continue;
                dl.push_back(make_int4(dx, dy, dz, (dz * SY + dy) * SX + dx));
                for (double v : g) gv.push_back((T)v);
            }
    MOT_TRY(dalloc(D.d, sizeof(int4) * std::max<size_t>(1, dl.size())));
    MOT_TRY(dalloc(D.g, sizeof(T) * std::max<size_t>(1, gv.size())));
    if (!dl.empty()) {
        MOT_CUDA_TRY(cudaMemcpy(D.d.p, dl.data(), sizeof(int4) * dl.size(), cudaMemcpyHostToDevice));
        MOT_CUDA_TRY(cudaMemcpy(D.g.p, gv.data(), sizeof(T) * gv.size(), cudaMemcpyHostToDevice));
    }
    D.fp32 = fp32;
    D.SX = SX;
    D.SY = SY;
    D.nd = (int)dl.size();
    return MOT_OK;
}

template <typename T> mot_status z0_direct(mot_problem *p, const T *x, T *y, int nrhs, cudaStream_t st) {
    int t[3];
    const int R[3] = {p->lags[0].R[0], p->lags[0].R[1], p->lags[0].R[2]};
    if (!direct_tile(p, sizeof(T), t)) {  // haloed tile too large for shared memory: unstaged kernel
        MOT_TRY(direct_list<T>(p, 0, 0));
        const long nv = (long)p->N[0] * p->N[1] * p->N[2];
        count_launch();
        k_z0_direct_g<T><<<dim3((unsigned)std::min<long>((nv + 255) / 256, 16L * p->ctx->sms), nrhs), 256, 0, st>>>(
            x, y, eps_of<T>(p), (const int4 *)p->direct.d.p, (const T *)p->direct.g.p, p->direct.nd, p->N[0],
            p->N[1], p->N[2], (T)p->opt.delta);
        MOT_CHECK_LAUNCH();
        return MOT_OK;
    }
    const int SX = t[0] + 2 * R[0], SY = t[1] + 2 * R[1], SZ = t[2] + 2 * R[2];
    MOT_TRY(direct_list<T>(p, SX, SY));
    const size_t smem = 3 * sizeof(T) * (size_t)SX * SY * SZ;
    MOT_TRY(allow_smem<k_z0_direct<T>>());
    const int tiles = ((p->N[0] + t[0] - 1) / t[0]) * ((p->N[1] + t[1] - 1) / t[1]) * ((p->N[2] + t[2] - 1) / t[2]);
    count_launch();
    k_z0_direct<T><<<dim3(tiles, nrhs), dim3(t[0], t[1], t[2]), smem, st>>>(
        x, y, eps_of<T>(p), (const int4 *)p->direct.d.p, (const T *)p->direct.g.p, p->direct.nd, R[0], R[1], R[2],
        p->N[0], p->N[1], p->N[2], (T)p->opt.delta);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}
}  // namespace

extern "C" {

const char *mot_last_error(void) { return get_error(); }

mot_status mot_ctx_create(int device, void *cuda_stream, mot_ctx **out) {
    if (!out) MOT_FAIL(MOT_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        MOT_FAIL(MOT_ECUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
    }
    if (device < 0 || device >= ndev) MOT_FAIL(MOT_EINVAL, "device index out of range");
    MOT_CUDA_TRY(cudaSetDevice(device));
    mot_ctx *c = new mot_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    // NULL is the CUDA legacy default stream (the stream PyTorch uses by default)
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
    *out = c;
    return MOT_OK;
}

void mot_ctx_destroy(mot_ctx *c) {
    if (!c) return;
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

mot_status mot_table_host(double rho, int lag, const int32_t R[3], double *g_out) {
    if (!(rho > 0.0) || !std::isfinite(rho)) MOT_FAIL(MOT_EINVAL, "rho must be finite and > 0");
    if (lag < 0) MOT_FAIL(MOT_EINVAL, "lag < 0");
    if (!R || !g_out) MOT_FAIL(MOT_EINVAL, "R or g_out is NULL");
    for (int i = 0; i < 3; ++i)
        if (R[i] < 0 || R[i] > 4096) MOT_FAIL(MOT_EINVAL, "table extent out of range");
    const HostRule &hr = host_rule();
    gk::Rule q = {hr.x, hr.w, kGLN}, q8 = {hr.x + kGLN, hr.w + kGLN, kGL8};
    int S[3] = {R[0], R[1], R[2]};
    std::sort(S, S + 3);
    ItemSet is;
    if (!build_items(rho, S, lag, lag, is))
        MOT_FAIL(MOT_EUNSUPPORTED, "time step too small for the lag-table quadrature (rho < 0.25)");
    std::vector<double> FM(std::max(1L, is.fm_len), 0.0), BM(std::max(1L, is.bm_len), 0.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < (long)is.faces.size(); ++i) {
        const FaceRec &f = is.faces[i];
        if (f.nj > 0) gk::face_moments(q, rho, (double)f.c, (double)f.a, (double)f.b, f.jlo, f.nj, &FM[f.off]);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < (long)is.tri.size(); ++i) {
        const TripleRec &t = is.tri[i];
        if (t.nj <= 0) continue;
        double *o = &BM[t.off];
        gk::box_moments(q, q8, rho, t.x, t.y, t.z, t.jlo, t.nj, o);
        gk::box_moments(q, q8, rho, t.x, t.z, t.y, t.jlo, t.nj, o + 3 * t.nj);
        gk::box_moments(q, q8, rho, t.y, t.z, t.x, t.jlo, t.nj, o + 6 * t.nj);
    }
    std::vector<double> A6(6 * std::max<size_t>(1, is.items.size()));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)is.items.size(); ++i)
        combine_item(is.items[i], is.tri.data(), is.faces.data(), FM.data(), BM.data(), &A6[6 * i]);
    std::vector<int> map;
    lag_map(is, lag, map);
    int Ri[3] = {R[0], R[1], R[2]};
    long on = (long)(Ri[0] + 1) * (Ri[1] + 1) * (Ri[2] + 1);
    std::vector<double> oct(6 * on);
    for (int dz = 0; dz <= Ri[2]; ++dz)
        for (int dy = 0; dy <= Ri[1]; ++dy)
            for (int dx = 0; dx <= Ri[0]; ++dx) {
                double g6[6];
                expand_one(A6.data(), map.data(), is.Rm, dx, dy, dz, g6);
                long oi = ((long)dz * (Ri[1] + 1) + dy) * (Ri[0] + 1) + dx;
                for (int c = 0; c < 6; ++c) oct[c * on + oi] = g6[c];
            }
    octant_to_full(oct, Ri, g_out);
    return MOT_OK;
}

mot_status mot_problem_create(mot_ctx *ctx, const int32_t n[3], double h, const double *eps_r, double alpha,
                              const mot_options *opt, mot_problem **out) {
    if (!ctx || !n || !eps_r || !out) MOT_FAIL(MOT_EINVAL, "NULL argument");
    *out = nullptr;
    for (int i = 0; i < 3; ++i)
        if (n[i] < 1 || n[i] > 4096) MOT_FAIL(MOT_EINVAL, "grid size out of range [1, 4096]");
    if (!(h > 0.0) || !std::isfinite(h)) MOT_FAIL(MOT_EINVAL, "h must be finite and > 0");
    if (!(alpha > 0.0) || !std::isfinite(alpha) || alpha > 1e4) MOT_FAIL(MOT_EINVAL, "alpha must be in (0, 1e4]");
    long nv = (long)n[0] * n[1] * n[2];
    for (long i = 0; i < nv; ++i)
        if (!std::isfinite(eps_r[i]) || eps_r[i] < 1.0) MOT_FAIL(MOT_EINVAL, "eps_r must be finite and >= 1");
    mot_options o = {0.0, 500, 1e-6, 6, 0.0, 0, 2, 1, 1};
    if (opt) o = *opt;
    if (!std::isfinite(o.delta)) MOT_FAIL(MOT_EINVAL, "delta must be finite");
    if (o.maxit < 1) MOT_FAIL(MOT_EINVAL, "maxit < 1");
    if (o.guess < 0 || o.guess > 2) MOT_FAIL(MOT_EINVAL, "guess must be 0, 1 or 2");
    if (o.graph < 0 || o.graph > 2) MOT_FAIL(MOT_EINVAL, "graph must be 0, 1 or 2");
    if (o.autotune != 0 && o.autotune != 1) MOT_FAIL(MOT_EINVAL, "autotune must be 0 or 1");
    MOT_CUDA_TRY(cudaSetDevice(ctx->device));
    mot_problem *p = new mot_problem();
    p->ctx = ctx;
    p->opt = o;
    for (int i = 0; i < 3; ++i) p->N[i] = n[i];
    p->h = h;
    p->alpha = alpha;
    p->rho = alpha / sqrt(3.0);
    p->dt = alpha * h / (kC0 * sqrt(3.0));
    double rmax = sqrt((double)n[0] * n[0] + (double)n[1] * n[1] + (double)n[2] * n[2]);
    p->ell = (int)ceil(rmax / p->rho - 1e-12) + 2;
    p->r0 = lag_reach(0, p->rho);
    for (int i = 0; i < 3; ++i) {
        int r = std::min(p->r0, n[i] - 1);
        p->M0[i] = smooth235(n[i] + r);
        p->Mh[i] = smooth235(std::max(1, 2 * n[i] - 1));
        p->K0[i] = p->M0[i] / 2 + 1;
        p->Kh[i] = p->Mh[i] / 2 + 1;
    }
    p->H0 = p->K0[0];
    p->Hh = p->Kh[0];
    p->eps_host.assign(eps_r, eps_r + nv);
    p->lags.resize(p->ell + 1);
    mot_status s;
    auto fail = [&](mot_status st) {
        mot_problem_destroy(p);
        return st;
    };
    if ((s = dalloc(p->eps, sizeof(double) * nv)) != MOT_OK) return fail(s);
    if (cudaMemcpyAsync(p->eps.p, eps_r, sizeof(double) * nv, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
        return fail(MOT_ECUDA);
    {
        std::vector<float> e32(eps_r, eps_r + nv);
        if ((s = dalloc(p->eps32, sizeof(float) * nv)) != MOT_OK) return fail(s);
        if (cudaMemcpy(p->eps32.p, e32.data(), sizeof(float) * nv, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(MOT_ECUDA);
    }
    {
        const HostRule &hr = host_rule();
        if ((s = dalloc(p->glx, sizeof(double) * (kGLN + kGL8))) != MOT_OK) return fail(s);
        if ((s = dalloc(p->glw, sizeof(double) * (kGLN + kGL8))) != MOT_OK) return fail(s);
        cudaMemcpyAsync(p->glx.p, hr.x, sizeof(double) * (kGLN + kGL8), cudaMemcpyHostToDevice, ctx->stream);
        cudaMemcpyAsync(p->glw.p, hr.w, sizeof(double) * (kGLN + kGL8), cudaMemcpyHostToDevice, ctx->stream);
    }
    for (int i = 0; i < 3; ++i)
        if (!get_tw(p, p->M0[i]) || !get_tw(p, p->Mh[i])) {
            set_error("FFT twiddle setup failed");
            return fail(MOT_ECUDA);
        }
    if ((s = compute_lag_octants(p, 0, 0)) != MOT_OK) return fail(s);
    if ((s = build_Z0_spectrum(p)) != MOT_OK) return fail(s);
    *out = p;
    return MOT_OK;
}

mot_status mot_problem_info_get(const mot_problem *p, mot_problem_info *info) {
    if (!p || !info) MOT_FAIL(MOT_EINVAL, "NULL argument");
    for (int i = 0; i < 3; ++i) {
        info->n[i] = p->N[i];
        info->M0[i] = p->M0[i];
        info->Mh[i] = p->Mh[i];
    }
    info->r0 = p->r0;
    info->ell = p->ell;
    info->rho = p->rho;
    info->dt = p->dt;
    return MOT_OK;
}

void mot_problem_destroy(mot_problem *p) {
    if (!p) return;
    cudaSetDevice(p->ctx->device);
    cudaStreamSynchronize(p->ctx->stream);
    dfree(p->eps);
    dfree(p->eps32);
    dfree(p->direct.d);
    dfree(p->direct.g);
    for (auto *t : p->tws) {
        dfree(t->tw64);
        dfree(t->tw32);
        dfree(t->twdf);
        delete t;
    }
    for (auto &L : p->lags) dfree(L.oct);
    dfree(p->L0_64);
    dfree(p->L0_32);
    dfree(p->L0_df);
    // shared spectra are released with the holder, not freed here
    if (p->lh_hold[0]) p->Lh_64.p = nullptr;
    if (p->lh_hold[1]) p->Lh_32.p = nullptr;
    if (p->lh_hold[2]) p->Lh_df.p = nullptr;
    for (auto &h : p->lh_hold) h.reset();
    dfree(p->Lh_64);
    dfree(p->Lh_32);
    dfree(p->Lh_df);
    dfree(p->glx);
    dfree(p->glw);
    dfree(p->wsA);
    dfree(p->wsB);
    delete p;
}

mot_status mot_apply_Z0(mot_problem *p, const void *x_dev, void *y_dev, int nrhs, int dtype) {
    if (!p || !x_dev || !y_dev) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (nrhs < 1) MOT_FAIL(MOT_EINVAL, "nrhs < 1");
    if (dtype != MOT_F64 && dtype != MOT_F32 && dtype != MOT_F64DF)
        MOT_FAIL(MOT_EINVAL, "dtype must be MOT_F64, MOT_F32 or MOT_F64DF");
    if (x_dev == y_dev) MOT_FAIL(MOT_EINVAL, "x and y must not overlap");
    if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 15u)
        MOT_FAIL(MOT_EINVAL, "x and y must be 16-byte aligned");
    MOT_CUDA_TRY(cudaSetDevice(p->ctx->device));
    size_t a, b;
    z0_ws_bytes(p, nrhs, dtype == MOT_F32 ? sizeof(float2) : sizeof(double2), &a, &b);
    MOT_TRY(dalloc(p->wsA, a));
    MOT_TRY(dalloc(p->wsB, b));
    const long pr = (long)p->N[2] * p->N[1];
    const Sched *sc = nullptr;
    if (dtype == MOT_F64) {
        MOT_TRY(schedule_for<double>(p, nrhs, &sc));
        SchedScope scope(sc);
        EpiZ0<double, double> e = {(const double *)x_dev, (double *)y_dev, eps_of<double>(p), pr, p->N[0],
                                   p->opt.delta};
        return z0_product<double, double>(p, (const double *)x_dev, nrhs, p->wsA.p, p->wsB.p, e, p->ctx->stream);
    }
    if (dtype == MOT_F64DF) {
        // the FP64 schedule's shapes (same element size), without a tuning pass of its own
        MOT_TRY(schedule_for<double>(p, nrhs, &sc));
        SchedScope scope(sc);
        EpiZ0DF e = {(const double *)x_dev, (double *)y_dev, eps_of<double>(p), pr, p->N[0], p->opt.delta};
        return z0_product<double, dfl>(p, (const double *)x_dev, nrhs, p->wsA.p, p->wsB.p, e, p->ctx->stream);
    }
    MOT_TRY(schedule_for<float>(p, nrhs, &sc));
    SchedScope scope(sc);
    EpiZ0<float, float> e = {(const float *)x_dev, (float *)y_dev, eps_of<float>(p), pr, p->N[0],
                             (float)p->opt.delta};
    return z0_product<float, float>(p, (const float *)x_dev, nrhs, p->wsA.p, p->wsB.p, e, p->ctx->stream);
}

mot_status mot_apply_Z0_direct(mot_problem *p, const void *x_dev, void *y_dev, int nrhs, int dtype) {
    if (!p || !x_dev || !y_dev) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (nrhs < 1 || nrhs > 65535) MOT_FAIL(MOT_EINVAL, "nrhs out of range [1, 65535]");
    if (dtype != MOT_F64 && dtype != MOT_F32) MOT_FAIL(MOT_EINVAL, "dtype must be MOT_F64 or MOT_F32");
    if (x_dev == y_dev) MOT_FAIL(MOT_EINVAL, "x and y must not overlap");
    MOT_CUDA_TRY(cudaSetDevice(p->ctx->device));
    if (dtype == MOT_F64) return z0_direct<double>(p, (const double *)x_dev, (double *)y_dev, nrhs, p->ctx->stream);
    return z0_direct<float>(p, (const float *)x_dev, (float *)y_dev, nrhs, p->ctx->stream);
}

mot_status mot_problem_schedule(const mot_problem *p, int nrhs, int dtype, mot_schedule *out) {
    if (!p || !out) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (dtype != MOT_F64 && dtype != MOT_F32) MOT_FAIL(MOT_EINVAL, "dtype must be MOT_F64 or MOT_F32");
    for (auto &t : p->tuned)
        if (t.nrhs == nrhs && t.fp32 == (dtype == MOT_F32)) {
            *out = t.info;
            return MOT_OK;
        }
    MOT_FAIL(MOT_EINVAL, "no tuned schedule for this (nrhs, dtype)");
}

mot_status mot_kernel_table(mot_problem *p, int lag, double *g_out, int32_t R_out[3]) {
    if (!p || !R_out) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (lag < 0 || lag > p->ell) MOT_FAIL(MOT_EINVAL, "lag out of range [0, ell]");
    MOT_CUDA_TRY(cudaSetDevice(p->ctx->device));
    LagTable &L = p->lags[lag];
    if (!L.ready) MOT_TRY(compute_lag_octants(p, lag, lag));
    for (int i = 0; i < 3; ++i) R_out[i] = L.R[i];
    if (!g_out) return MOT_OK;
    long on = (long)(L.R[0] + 1) * (L.R[1] + 1) * (L.R[2] + 1);
    std::vector<double> oct(6 * on);
    MOT_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
    MOT_CUDA_TRY(cudaMemcpy(oct.data(), L.oct.p, sizeof(double) * 6 * on, cudaMemcpyDeviceToHost));
    octant_to_full(oct, L.R, g_out);
    return MOT_OK;
}

mot_status mot_set_kernel_table(mot_problem *p, int lag, const double *g, const int32_t R[3]) {
    if (!p || !g || !R) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (lag < 0 || lag > p->ell) MOT_FAIL(MOT_EINVAL, "lag out of range [0, ell]");
    if (lag >= 1 && (p->hist64 || p->hist32 || p->histdf)) MOT_FAIL(MOT_EINVAL, "history tables already in use; set them before mot_run_create");
    for (int i = 0; i < 3; ++i)
        if (R[i] < 0 || R[i] > 4096) MOT_FAIL(MOT_EINVAL, "table extent out of range");
    MOT_CUDA_TRY(cudaSetDevice(p->ctx->device));
    int nx = 2 * R[0] + 1, ny = 2 * R[1] + 1, nz = 2 * R[2] + 1;
    long n3 = (long)nx * ny * nz;
    if (!finite_all(g, 6 * n3)) MOT_FAIL(MOT_EINVAL, "table has non-finite entries");
    LagTable &L = p->lags[lag];
    int Rc[3];
    for (int i = 0; i < 3; ++i) Rc[i] = std::min<int>(R[i], p->N[i] - 1);
    if (lag == 0)
        for (int i = 0; i < 3; ++i)
            if (Rc[i] > p->M0[i] - p->N[i]) MOT_FAIL(MOT_EINVAL, "lag-0 table reaches beyond the padded grid M0 - N");
    long on = (long)(Rc[0] + 1) * (Rc[1] + 1) * (Rc[2] + 1);
    std::vector<double> oct(6 * on);
    for (int c = 0; c < 6; ++c)
        for (int dz = 0; dz <= Rc[2]; ++dz)
            for (int dy = 0; dy <= Rc[1]; ++dy)
                for (int dx = 0; dx <= Rc[0]; ++dx) {
                    long fi = ((long)(dz + R[2]) * ny + (dy + R[1])) * nx + (dx + R[0]);
                    oct[c * on + ((long)dz * (Rc[1] + 1) + dy) * (Rc[0] + 1) + dx] = g[c * n3 + fi];
                }
    MOT_TRY(dalloc(L.oct, sizeof(double) * 6 * on));
    MOT_CUDA_TRY(cudaMemcpy(L.oct.p, oct.data(), sizeof(double) * 6 * on, cudaMemcpyHostToDevice));
    for (int i = 0; i < 3; ++i) L.R[i] = Rc[i];
    L.ready = true;
    L.override_ = true;
    if (lag == 0) MOT_TRY(build_Z0_spectrum(p));
    return MOT_OK;
}

}  // extern "C"

// ============================================================================
// marching runs
// ============================================================================
namespace {

// Krylov vector slots
enum { kRS = 0, kW, kY1, kY2, kV, kD, kAY1, kAY2, kX, kB };

template <typename V> struct KrylovView {
    V *v[10];
    TfqmrScal *sc;
    double *p1, *p2, *p3;
};

template <typename V> KrylovView<V> kview(mot_run *r) {
    KrylovView<V> k;
    for (int i = 0; i < 10; ++i) k.v[i] = (V *)r->kv[i].p;
    k.sc = (TfqmrScal *)r->scal.p;
    k.p1 = (double *)r->part1.p;
    k.p2 = (double *)r->part2.p;
    k.p3 = (double *)r->part3.p;
    return k;
}

template <typename V> mot_status mvp(mot_run *r, const V *x, V *y, cudaStream_t st) {
    mot_problem *p = r->p;
    EpiZ0<V, V> e = {x, y, eps_of<V>(p), (long)p->N[2] * p->N[1], p->N[0], (V)p->opt.delta};
    return z0_product<V, V>(p, x, r->B, p->wsA.p, p->wsB.p, e, st);
}

// x0 = 2 J_{n-1} - J_{n-2} in J, and J_{n-1} saved into J2
__global__ void k_extrapolate(double *__restrict__ J, double *__restrict__ J2, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        double a = J[i];
        J[i] = 2.0 * a - J2[i];
        J2[i] = a;
    }
}

// x0 = 3 J_{n-1} - 3 J_{n-2} + J_{n-3} in J (the quadratic through the last
// three currents), J_{n-1} saved into J2 and J_{n-2} into J3
__global__ void k_extrapolate2(double *__restrict__ J, double *__restrict__ J2, double *__restrict__ J3, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double a = J[i], b = J2[i];
        J[i] = 3.0 * (a - b) + J3[i];
        J3[i] = b;
        J2[i] = a;
    }
}

// the step's initial guess in J from the saved currents (options.guess)
mot_status launch_guess(mot_run *r, long n, cudaStream_t st) {
    const int g = r->p->opt.guess;
    if (g == 0) return MOT_OK;
    count_launch();
    if (g == 1) k_extrapolate<<<grid_for(n), 256, 0, st>>>((double *)r->J.p, (double *)r->J2.p, n);
    else k_extrapolate2<<<grid_for(n), 256, 0, st>>>((double *)r->J.p, (double *)r->J2.p, (double *)r->J3.p, n);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

template <typename T> __global__ void k_sub(T *__restrict__ w, const T *__restrict__ b, const T *__restrict__ a, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        w[i] = b[i] - a[i];
}

// Z0 y1 with y1 = w + beta y2 formed by the forward plane pass (one vector
// pass fewer); where the planes do not fit, y1 is formed first
template <typename V> mot_status mvp_y1(mot_run *r, cudaStream_t st) {
    mot_problem *p = r->p;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    KrylovView<V> k = kview<V>(r);
    if (!z0_planes_fit<V>(p)) {
        if (!p->capturing) p->kt.begin(st, MOT_K_VEC);
        count_launch();
        k_tfqmr_y1<V><<<dim3(grid_for(L), r->B), 256, 0, st>>>(k.v[kY1], k.v[kW], k.v[kY2], k.sc, L);
        MOT_CHECK_LAUNCH();
        if (!p->capturing) p->kt.end(st);
        return mvp<V>(r, k.v[kY1], k.v[kAY1], st);
    }
    SrcY1<V> src = {k.v[kY1], k.v[kW], k.v[kY2], k.sc, L};
    EpiZ0<V, V> e = {k.v[kY1], k.v[kAY1], eps_of<V>(p), (long)p->N[2] * p->N[1], p->N[0], (V)p->opt.delta};
    return z0_product_src<SrcY1<V>, V, V>(p, src, (const V *)nullptr, r->B, p->wsA.p, p->wsB.p, e, st);
}

// one TFQMR iteration (two half steps, two Z0 products) on stream st, ending
// with the next alpha and the loop test (graph handle h if use_h, else ctl[2]).
// Where the product runs as plane passes the vector updates ride in them
// (six kernels); otherwise separate vector kernels (nine or ten).
template <typename V>
mot_status tfqmr_body(mot_run *r, V *x, cudaStream_t st, cudaGraphConditionalHandle h, int use_h) {
    mot_problem *p = r->p;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    KrylovView<V> k = kview<V>(r);
    unsigned *ctr = (unsigned *)r->ctr.p;
    dim3 gr(kRedBlocks, r->B);
    if (z0_planes_fit<V>(p)) {
        const int P = 3 * p->N[2];
        const V *eps = eps_of<V>(p);
        SrcHalfA<V> sa = {x, k.v[kW], k.v[kD], k.v[kY2], k.v[kY1], k.v[kAY1], k.v[kV], k.sc, L, k.p1, P, ctr};
        EpiHalfB<V> eb = {k.v[kY2], k.v[kAY2], eps, x, k.v[kW], k.v[kD], k.v[kRS], k.sc, k.p1, k.p2, P, ctr + 1,
                          (V)p->opt.delta};
        MOT_TRY((z0_product_src<SrcHalfA<V>, V, V>(p, sa, (const V *)nullptr, r->B, p->wsA.p, p->wsB.p, eb, st)));
        SrcY1<V> s1 = {k.v[kY1], k.v[kW], k.v[kY2], k.sc, L};
        EpiV<V> ev = {k.v[kY1], k.v[kAY1], eps, k.v[kV], k.v[kAY2], k.v[kRS], k.sc, k.p3, P, ctr + 2,
                      (int *)r->ctl.p, h, use_h, 0, (V)p->opt.delta};
        MOT_TRY((z0_product_src<SrcY1<V>, V, V>(p, s1, (const V *)nullptr, r->B, p->wsA.p, p->wsB.p, ev, st)));
        return MOT_OK;
    }
    const bool timed = !p->capturing;
    if (timed) p->kt.begin(st, MOT_K_VEC);
    count_launch();
    k_tfqmr_half_a<V><<<gr, kRedThreads, 0, st>>>(x, k.v[kW], k.v[kD], k.v[kY2], k.v[kY1], k.v[kAY1], k.v[kV], k.sc,
                                                   L, k.p1, ctr);
    MOT_CHECK_LAUNCH();
    if (timed) p->kt.end(st);
    MOT_TRY(mvp<V>(r, k.v[kY2], k.v[kAY2], st));
    if (timed) p->kt.begin(st, MOT_K_VEC);
    count_launch();
    k_tfqmr_half_b<V><<<gr, kRedThreads, 0, st>>>(x, k.v[kW], k.v[kD], k.v[kY2], k.v[kAY2], k.v[kRS], k.sc, L, k.p1,
                                                   k.p2, ctr + 1);
    MOT_CHECK_LAUNCH();
    if (timed) p->kt.end(st);
    MOT_TRY(mvp_y1<V>(r, st));
    if (timed) p->kt.begin(st, MOT_K_VEC);
    count_launch();
    k_tfqmr_v<V><<<gr, kRedThreads, 0, st>>>(k.v[kV], k.v[kAY1], k.v[kAY2], k.v[kRS], k.sc, L, k.p3, ctr + 2,
                                              (int *)r->ctl.p, h, use_h);
    MOT_CHECK_LAUNCH();
    if (timed) p->kt.end(st);
    return MOT_OK;
}

// build the graph: while (cond) { tfqmr_body }, the body setting cond
template <typename V> mot_status build_loop_graph(mot_run *r, V *x, LoopGraph &G) {
    mot_problem *p = r->p;
    cudaGraph_t g = nullptr;
    MOT_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    MOT_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    MOT_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const unsigned long long l0 = g_launches.load();
    p->capturing = true;
    MOT_CUDA_TRY(cudaStreamBeginCaptureToGraph(r->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    mot_status s = tfqmr_body<V>(r, x, r->cap, h, 1);
    cudaGraph_t out = nullptr;
    cudaError_t ce = cudaStreamEndCapture(r->cap, &out);
    p->capturing = false;
    const unsigned long long l1 = g_launches.load();
    g_launches.fetch_sub(l1 - l0);  // captured, not launched
    if (s != MOT_OK) {
        cudaGraphDestroy(g);
        return s;
    }
    if (ce != cudaSuccess) {
        cudaGraphDestroy(g);
        MOT_FAIL(MOT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    }
    cudaError_t ie = cudaGraphInstantiate(&G.exec, g, 0);
    if (ie != cudaSuccess) {
        cudaGraphDestroy(g);
        MOT_FAIL(MOT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    }
    G.graph = g;
    G.x = x;
    G.body_kernels = (int)(l1 - l0);
    return MOT_OK;
}

// the solve start from x0 = 0 runs as two kernels plus a product (the plane
// passes carry v = Z0 y1 and the first alpha)
template <typename V> bool fused_start(const mot_problem *p) { return z0_planes_fit<V>(p); }

// start of a solve on st: r0 = rhs - Z0 x0 into w (x0 = 0 if zero_x0), y1 = r* =
// w, d = 0, tau and rho, x = 0 where rhs = 0, v = Z0 y1 and the first alpha.
// With src64 (zero_x0 and fused_start only) the right-hand side is 2^-e src64,
// e from the squared norms n2 (the mixed form's correction solve), and rhs is
// not read.  *mvps: products applied.
// the adaptive inner tolerance of the mixed refinement (InnerTol): the FP32
// correction solve is given 0.3 of the outer tolerance, the rest left to its
// rounding; MOTJVIE_INNER_ADAPT=0 keeps inner_tol fixed (timing comparisons)
mot_status dev_norms2(mot_run *r, const double *v, double *out, cudaStream_t st);

// outer tolerance of the refined precisions: the mixed path's 1e-6, the
// double-float path's FP64-level 1e-11 (options.tol overrides)
inline double outer_tol(const mot_run *r) {
    const double t = r->p->opt.tol;
    return t > 0 ? t : (r->prec == MOT_FP64DF ? 1e-11 : 1e-6);
}

// the outer residual r = b - Z0 J of the refinement: the product's FFT in FP32
// (MOT_MIXED) or in double-float (MOT_FP64DF), its epilogue in FP64
mot_status residual_product(mot_run *r, cudaStream_t st) {
    mot_problem *p = r->p;
    const long pr = (long)p->N[2] * p->N[1];
    EpiResidual e = {(const double *)r->J.p, (const double *)r->b.p, (double *)r->r.p, (const double *)p->eps.p, pr,
                     p->N[0], p->opt.delta};
    if (r->prec == MOT_FP64DF)
        return z0_product<double, dfl>(p, (const double *)r->J.p, r->B, p->wsA.p, p->wsB.p, e, st);
    return z0_product<double, float>(p, (const double *)r->J.p, r->B, p->wsA.p, p->wsB.p, e, st);
}

inline InnerTol inner_tol_for(mot_run *r, const double *ro2, double tol) {
    static const bool off = getenv("MOTJVIE_INNER_ADAPT") && atoi(getenv("MOTJVIE_INNER_ADAPT")) == 0;
    InnerTol it;
    if (off) return it;
    it.bo2 = (const double *)r->b2.p;
    it.ro2 = ro2;
    it.otol = 0.3 * tol;
    return it;
}

template <typename V>
mot_status tfqmr_start(mot_run *r, V *x, const V *rhs, bool zero_x0, double tol, cudaStream_t st, int *mvps,
                       const double *src64 = nullptr, const double *n2 = nullptr, InnerTol itol = InnerTol{}) {
    mot_problem *p = r->p;
    const int B = r->B;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    const long n = L * B;
    KrylovView<V> k = kview<V>(r);
    dim3 gv(grid_for(L), B), gr(kRedBlocks, B);
    *mvps = 1;
    if (src64 && !(zero_x0 && fused_start<V>(p))) MOT_FAIL(MOT_EINVAL, "scaled start needs the fused path");
    if (zero_x0 && fused_start<V>(p)) {
        unsigned *ctr = (unsigned *)r->ctr.p;
        const int stag = sizeof(V) == 4 ? 1 : 0;  // FP32 solves stop at stagnation
        count_launch();
        if (src64)
            k_tfqmr_start_zero<V, double><<<gr, kRedThreads, 0, st>>>(src64, n2, x, k.v[kW], k.v[kY1], k.v[kRS],
                                                                      k.v[kD], L, k.p1, k.sc, tol, stag, ctr + 3,
                                                                      itol);
        else
            k_tfqmr_start_zero<V, V><<<gr, kRedThreads, 0, st>>>(rhs, nullptr, x, k.v[kW], k.v[kY1], k.v[kRS], k.v[kD],
                                                                 L, k.p1, k.sc, tol, stag, ctr + 3, itol);
        MOT_CHECK_LAUNCH();
        EpiV<V> ev = {k.v[kY1], k.v[kAY1], eps_of<V>(p), k.v[kV], k.v[kAY2], k.v[kRS], k.sc, k.p3, 3 * p->N[2],
                      ctr + 2, (int *)r->ctl.p, cudaGraphConditionalHandle{}, 0, 1, (V)p->opt.delta};
        return z0_product<V, V>(p, (const V *)k.v[kY1], B, p->wsA.p, p->wsB.p, ev, st);
    }
    if (zero_x0) {
        MOT_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(V) * n, st));
        MOT_CUDA_TRY(cudaMemcpyAsync(k.v[kW], rhs, sizeof(V) * n, cudaMemcpyDeviceToDevice, st));
    } else {
        MOT_TRY(mvp<V>(r, x, k.v[kAY1], st));
        *mvps = 2;
        count_launch();
        k_sub<V><<<grid_for(n), 256, 0, st>>>(k.v[kW], rhs, k.v[kAY1], n);
        MOT_CHECK_LAUNCH();
    }
    MOT_CUDA_TRY(cudaMemcpyAsync(k.v[kY1], k.v[kW], sizeof(V) * n, cudaMemcpyDeviceToDevice, st));
    MOT_CUDA_TRY(cudaMemcpyAsync(k.v[kRS], k.v[kW], sizeof(V) * n, cudaMemcpyDeviceToDevice, st));
    MOT_CUDA_TRY(cudaMemsetAsync(k.v[kD], 0, sizeof(V) * n, st));
    count_launch();
    k_dot_part<V, V><<<gr, kRedThreads, 0, st>>>(k.v[kW], k.v[kW], L, k.p1);
    count_launch();
    k_dot_part<V, V><<<gr, kRedThreads, 0, st>>>(rhs, rhs, L, k.p2);
    count_launch();
    // FP32 inner solves stop at stagnation; the FP64 solve runs to tol or maxit
    k_tfqmr_init<<<B, 32, 0, st>>>(k.sc, k.p1, k.p2, tol, sizeof(V) == 4 ? 1 : 0, itol);
    count_launch();
    k_tfqmr_zero_rhs<V><<<gv, 256, 0, st>>>(x, k.sc, L);
    count_launch();
    k_tfqmr_zero_done<<<(B + 255) / 256, 256, 0, st>>>(k.sc, B);
    MOT_CHECK_LAUNCH();
    MOT_TRY(mvp<V>(r, k.v[kY1], k.v[kAY1], st));
    MOT_CUDA_TRY(cudaMemcpyAsync(k.v[kV], k.v[kAY1], sizeof(V) * n, cudaMemcpyDeviceToDevice, st));
    count_launch();
    k_dot_part<V, V><<<gr, kRedThreads, 0, st>>>(k.v[kRS], k.v[kV], L, k.p3);
    count_launch();
    k_tfqmr_alpha<<<B, 32, 0, st>>>(k.sc, k.p3);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

// TFQMR on Z0 y = rhs for the batch; x holds x0 on entry (x0 = 0 if zero_x0)
// and the solution on exit.  The iteration loop runs as one graph launch
// (graph option 0) or host-driven (graph option 2).
// iters_out: iterations (max over the batch); mvps_out: Z0 products applied.
template <typename V>
mot_status tfqmr(mot_run *r, V *x, const V *rhs, bool zero_x0, double tol, int maxit, int *iters_out,
                 bool *conv_out, int *mvps_out, const double *src64 = nullptr, const double *n2 = nullptr,
                 InnerTol itol = InnerTol{}) {
    mot_problem *p = r->p;
    cudaStream_t st = p->ctx->stream;
    const int B = r->B;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    KrylovView<V> k = kview<V>(r);
    dim3 gv(grid_for(L), B);
    int mvps = 0;
    MOT_TRY(tfqmr_start<V>(r, x, rhs, zero_x0, tol, st, &mvps, src64, n2, itol));
    int ctl_h[2] = {0, maxit};
    MOT_CUDA_TRY(cudaMemcpyAsync(r->ctl.p, ctl_h, sizeof(ctl_h), cudaMemcpyHostToDevice, st));
    if (p->opt.graph == 2) {
        // no graphs: the same body, its loop test read by the host
        int ctl_now[3] = {0, maxit, 1};
        while (ctl_now[2]) {
            MOT_TRY(tfqmr_body<V>(r, x, st, cudaGraphConditionalHandle{}, 0));
            MOT_CUDA_TRY(cudaMemcpyAsync(ctl_now, r->ctl.p, sizeof(ctl_now), cudaMemcpyDeviceToHost, st));
            MOT_CUDA_TRY(cudaStreamSynchronize(st));
        }
    } else {
        // the iteration loop: one graph launch
        LoopGraph &G = sizeof(V) == 8 ? r->loop64 : r->loop32;
        if (G.exec && G.x != (void *)x) MOT_FAIL(MOT_EINVAL, "solve graph bound to another vector");
        if (!G.exec) MOT_TRY(build_loop_graph<V>(r, x, G));
        MOT_CUDA_TRY(cudaGraphLaunch(G.exec, st));
    }
    count_launch();
    k_tfqmr_flush<V, V><<<gv, 256, 0, st>>>(x, k.v[kD], k.sc, L, 1);
    count_launch();
    k_tfqmr_settle<<<(B + 255) / 256, 256, 0, st>>>(k.sc, B, 1);
    MOT_CHECK_LAUNCH();
    std::vector<TfqmrScal> hs(B);
    MOT_CUDA_TRY(cudaMemcpyAsync(hs.data(), k.sc, sizeof(TfqmrScal) * B, cudaMemcpyDeviceToHost, st));
    MOT_CUDA_TRY(cudaMemcpyAsync(ctl_h, r->ctl.p, sizeof(ctl_h), cudaMemcpyDeviceToHost, st));
    MOT_CUDA_TRY(cudaStreamSynchronize(st));
    if (p->opt.graph != 2) {
        const LoopGraph &G = sizeof(V) == 8 ? r->loop64 : r->loop32;
        g_launches.fetch_add((unsigned long long)G.body_kernels * ctl_h[0]);
    }
    mvps += 2 * ctl_h[0];
    int mx = 0;
    bool conv = true;
    for (int b = 0; b < B; ++b) {
        mx = std::max(mx, (hs[b].m + 1) / 2);
        if (hs[b].conv == 0) conv = false;
    }
    *iters_out = mx;
    *conv_out = conv;
    *mvps_out = mvps;
    return MOT_OK;
}

template <typename T> void *ring_slot(mot_run *r, long s) {
    mot_problem *p = r->p;
    size_t slot = (size_t)r->B * 3 * p->Mh[2] * p->Mh[1] * p->Hh * sizeof(cplx<T>);
    return (char *)r->ring.p + slot * s;
}

// Jhat_n = F_Mh{J_n} into ring slot n mod ell
// nptr (graph mode): the slot index comes from device memory
template <typename T> mot_status ring_push(mot_run *r, cudaStream_t st, const long long *nptr = nullptr) {
    mot_problem *p = r->p;
    const int Nx = p->N[0], Ny = p->N[1], Nz = p->N[2];
    const int H = p->Hh, My = p->Mh[1], Mz = p->Mh[2];
    AxisTw *tx = get_tw(p, p->Mh[0]), *ty = get_tw(p, My), *tz = get_tw(p, Mz);
    using C = cplx<T>;
    C *A = (C *)r->wsAh.p, *Bf = (C *)r->wsBh.p;
    const long nrows = (long)r->B * 3 * Nz * Ny;
    if (xy_smem_bytes<T>(p->Mh[0], My, H, Ny) <= kSmemMax) {
        if (!p->capturing) p->kt.begin(st, MOT_K_FWD_RING);
        MOT_TRY((launch_xy_forward<SrcPlain<double>, T>(SrcPlain<double>{(const double *)r->J.p}, Bf, r->B * 3 * Nz, Nx,
                                                         Ny, H, tx, ty, st)));
        if (!p->capturing) p->kt.end(st);
    } else {
        if (!p->capturing) p->kt.begin(st, MOT_K_FWD_RING);
        if (x_forward_r<double, T>((const double *)r->J.p, A, nrows, Nx, Ny, tx, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_x_forward<double, T>((const double *)r->J.p, A, nrows, Nx, H, tx, st)));
        if (col_r<T, -1>(A, Bf, ty, H, Ny, My, r->B * 3 * Nz, (long)Ny * H, (long)My * H, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_axis<T, -1>(A, Bf, ty, H, Ny, My, r->B * 3 * Nz, 1, (long)Ny * H, 0, H, (long)My * H, 0, H, st)));
        if (!p->capturing) p->kt.end(st);
    }
    const long slot_elems = (long)r->B * 3 * Mz * My * H;
    C *slot = nptr ? (C *)r->ring.p : (C *)ring_slot<T>(r, r->n % p->ell);
    if (col_r<T, -1>(Bf, slot, tz, (int)((long)My * H), Nz, Mz, r->B * 3, (long)Nz * My * H, (long)Mz * My * H, st, nptr,
                     p->ell, slot_elems))
        MOT_CHECK_LAUNCH();
    else
        MOT_TRY((launch_axis<T, -1>(Bf, slot, tz, H, Nz, Mz, r->B * 3, My, (long)Nz * My * H, H, (long)My * H,
                                    (long)Mz * My * H, H, (long)My * H, st, nptr, p->ell, slot_elems)));
    return MOT_OK;
}

// b_n = E^i_n - eps T(dt) J_{n-1} + (eps - 1) sum_k G_k J_{n-k}
// the streaming history sum applies (grid within the 32-bit thread index)
bool hist_streaming(const mot_run *r) {
    const mot_problem *p = r->p;
    const long threads = (long)r->B * (p->Mh[2] / 2 + 1) * (p->Mh[1] / 2 + 1) * p->Hh;
    return r->hacc.p && r->hpart.p && threads < (1L << 31);
}

// blocks of bt threads for the streaming history sum, at most per_sm_x2 / 2 per SM
unsigned hist_blocks(const mot_run *r, long per_sm_x2, int bt = 256) {
    const mot_problem *p = r->p;
    const long threads = (long)r->B * (p->Mh[2] / 2 + 1) * (p->Mh[1] / 2 + 1) * p->Hh;
    return (unsigned)std::max<long>(1, std::min<long>((threads + bt - 1) / bt, per_sm_x2 * p->ctx->sms / 2));
}

// the step graph's side branch: one block of kHistSideThreads per SM leaves
// room beside it for the solve's kernels (MOTJVIE_HIST_SIDE_BPS2 = blocks per
// two SMs and MOTJVIE_HIST_SIDE_THREADS override, for sweeps)
long hist_side_per_sm_x2() {
    static const long f = getenv("MOTJVIE_HIST_SIDE_BPS2") ? std::max(1, atoi(getenv("MOTJVIE_HIST_SIDE_BPS2"))) : 1;
    return f;
}
int hist_side_threads() {
    static const int f = getenv("MOTJVIE_HIST_SIDE_THREADS") ? atoi(getenv("MOTJVIE_HIST_SIDE_THREADS")) : 256;
    return (f == 64 || f == 128 || f == 256) ? f : 256;
}

// the near accumulation's load mode: 0 plain loads + L2 prefetch, 1 evict-first +
// prefetch (default beside the solve), 2 evict-first only
int hist_side_mode() {
    static const int f = getenv("MOTJVIE_HIST_SIDE_MODE") ? atoi(getenv("MOTJVIE_HIST_SIDE_MODE")) : 1;
    return (f >= 0 && f <= 2) ? f : 1;
}

template <typename T> QSlots<T> qslots(mot_run *r, int flags) {
    const mot_problem *p = r->p;
    const long slot = (long)r->B * 3 * p->Mh[2] * p->Mh[1] * p->Hh;
    return QSlots<T>{(cplx<T> *)r->hpart.p, slot, r->hTB, flags};
}

// schedule of the time-blocked pass: 1 = the old part spread over the previous
// block's steps and the recent part at the block start (the block-start step is
// not held up by a whole pass: lower p99 step latency); 0 = one whole pass at the
// block start (fewer bytes).  MOTJVIE_HIST_SPREAD = 0 | 1 overrides the default.
inline bool hist_spread() {
    static const int f = getenv("MOTJVIE_HIST_SPREAD") ? atoi(getenv("MOTJVIE_HIST_SPREAD")) : 0;
    return f != 0;
}

// one part of the time-blocked pass (k_hist_block) for the block starting at
// m0, outputs t >= tlo, octant-point chunks [c_lo, c_hi) of hTB; with nptr the
// kernel takes its block and chunk from m = *nptr + dm (see k_hist_block)
template <typename T>
mot_status hist_block_pass(mot_run *r, cudaStream_t st, long m0, int tlo, int part, int c_lo, int c_hi,
                           const long long *nptr, int dm) {
    mot_problem *p = r->p;
    const int H = p->Hh, My = p->Mh[1], Mz = p->Mh[2];
    Octant oc = {Mz, My, p->Kh[2], p->Kh[1], H};
    const QSlots<T> q = qslots<T>(r, 0);
    const long points = (long)r->B * (Mz / 2 + 1) * (My / 2 + 1) * H;
    // points of the launch: all of them (recent part) or one chunk of hTB (old part)
    const int nchunks = nptr ? (part == kHistOld ? 1 : r->hTB) : c_hi - c_lo;
    const long lpoints = (points * nchunks + r->hTB - 1) / r->hTB;
    // blocks per SM (MOTJVIE_HIST_BLOCK_BPS overrides, for sweeps)
    static const long bps = getenv("MOTJVIE_HIST_BLOCK_BPS") ? std::max(1, atoi(getenv("MOTJVIE_HIST_BLOCK_BPS"))) : 32;
    const unsigned grid = (unsigned)std::max<long>(1, std::min<long>((lpoints + 31) / 32, bps * p->ctx->sms));
    const auto *ring = (const cplx<T> *)r->ring.p;
    if (r->hTB != (sizeof(T) == 4 ? 8 : 4)) MOT_FAIL(MOT_EINVAL, "time block does not match the history precision");
    // time block 8 (FP32) with two outputs per thread, 4 (FP64) with one: four thread groups
    constexpr int TB = sizeof(T) == 4 ? 8 : 4, TH = TB / 4;
    // L2 prefetch distance of the Lambda_k window in slots (MOTJVIE_HIST_LAM_PF; 0: none)
    static const int lpf = getenv("MOTJVIE_HIST_LAM_PF") ? std::max(0, atoi(getenv("MOTJVIE_HIST_LAM_PF"))) : 4;
    MOT_TRY(allow_smem<k_hist_block<T, TB, TH>>());
    count_launch();
    k_hist_block<T, TB, TH><<<grid, dim3(32, 4), hist_block_smem<T>(), st>>>(
        ring, Lh_of<T>(p), q.buf, q.slot, Mz, My, H, oc, r->B, p->ell, m0, tlo, part, c_lo, c_hi, nptr, dm, lpf);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

// the near accumulation of step m (lags 2 .. (m mod hTB) + 1, onto its slot)
template <typename T>
mot_status hist_near(mot_run *r, cudaStream_t st, long m, const long long *nptr, int dm, unsigned blocks, int bt,
                     int mode) {
    mot_problem *p = r->p;
    const int H = p->Hh, My = p->Mh[1], Mz = p->Mh[2];
    Octant oc = {Mz, My, p->Kh[2], p->Kh[1], H};
    const auto *ring = (const cplx<T> *)r->ring.p;
    const QSlots<T> q = qslots<T>(r, kQBase | kQAcc | kQNear);
    count_launch();
    if (mode == 1)
        k_hist_acc<T, 1><<<blocks, bt, 0, st>>>(ring, Lh_of<T>(p), nullptr, nullptr, Mz, My, H, oc, r->B, p->ell, m, 2,
                                                p->ell, nptr, dm, q);
    else if (mode == 2)
        k_hist_acc<T, 2><<<blocks, bt, 0, st>>>(ring, Lh_of<T>(p), nullptr, nullptr, Mz, My, H, oc, r->B, p->ell, m, 2,
                                                p->ell, nptr, dm, q);
    else
        k_hist_acc<T, 0><<<blocks, bt, 0, st>>>(ring, Lh_of<T>(p), nullptr, nullptr, Mz, My, H, oc, r->B, p->ell, m, 2,
                                                p->ell, nptr, dm, q);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

// the lags 2.. sum of step m = r->n into its slot, host-driven -- the kernels
// the step graph runs beside step m-1, in the same order: at a block start the
// recent part of the block, then chunk t = m mod hTB of the next block's old
// part, then the near accumulation of step m.  Stale slots (a new run, a loaded
// checkpoint) are rebuilt first: the block's old part (outputs t..), its recent
// part, the chunks 0..t-1 of the next block's old part.
template <typename T> mot_status hist_side_host(mot_run *r, cudaStream_t st, unsigned blocks, int bt, int mode) {
    const long m = r->n;
    const int TB = r->hTB, t = (int)(m % TB);
    const long m0 = m - t;
    if (!hist_spread()) {  // one whole pass at the block start
        if (t == 0 || r->q_stale) MOT_TRY(hist_block_pass<T>(r, st, m0, t, kHistAll, 0, TB, nullptr, 0));
        r->q_stale = false;
        return hist_near<T>(r, st, m, nullptr, 0, blocks, bt, mode);
    }
    if (r->q_stale) {
        MOT_TRY(hist_block_pass<T>(r, st, m0, t, kHistOld, 0, TB, nullptr, 0));
        MOT_TRY(hist_block_pass<T>(r, st, m0, t, kHistRecent, 0, TB, nullptr, 0));
        if (t > 0) MOT_TRY(hist_block_pass<T>(r, st, m0 + TB, 0, kHistOld, 0, t, nullptr, 0));
        r->q_stale = false;
    } else if (t == 0) {
        MOT_TRY(hist_block_pass<T>(r, st, m0, 0, kHistRecent, 0, TB, nullptr, 0));
    }
    MOT_TRY(hist_block_pass<T>(r, st, m0 + TB, 0, kHistOld, t, t + 1, nullptr, 0));
    return hist_near<T>(r, st, m, nullptr, 0, blocks, bt, mode);
}

// before a step-graph launch: the graph expects the lags 2.. sum of step n in its slot
mot_status hist_prime(mot_run *r, cudaStream_t st) {
    if (!hist_streaming(r) || r->hpart_ok) return MOT_OK;
    if (r->prec == MOT_MIXED) MOT_TRY(hist_side_host<float>(r, st, hist_blocks(r, 32), 256, 0));
    else if (r->prec == MOT_FP64DF) MOT_TRY(hist_side_host<dfl>(r, st, hist_blocks(r, 32), 256, 0));
    else MOT_TRY(hist_side_host<double>(r, st, hist_blocks(r, 32), 256, 0));
    r->hpart_ok = true;
    return MOT_OK;
}

template <typename T> mot_status history_rhs(mot_run *r, cudaStream_t st, const long long *nptr = nullptr) {
    mot_problem *p = r->p;
    const int Nx = p->N[0], Ny = p->N[1], Nz = p->N[2];
    const int H = p->Hh, My = p->Mh[1], Mz = p->Mh[2];
    const long nv = (long)Nx * Ny * Nz;
    AxisTw *tx = get_tw(p, p->Mh[0]), *ty = get_tw(p, My), *tz = get_tw(p, Mz);
    using C = cplx<T>;
    C *A = (C *)r->wsAh.p, *Bf = (C *)r->wsBh.p;
    const double t = (double)r->n * p->dt;
    count_launch();
    if (sizeof(T) == 4) {
        const long S = (long)Nx + Ny + Nz;
        const double *ts = (const double *)r->inctab.p;
        const float2 *ph = (const float2 *)(ts + S * r->B);
        const float *tsf = (const float *)(ph + S * r->B);
        const dim3 grid((unsigned)std::min<long>((long)Ny * Nz, 8L * p->ctx->sms), (unsigned)r->B);
        const int threads = std::min(256, (Nx + 31) / 32 * 32);
        k_incident_rows<<<grid, threads, 0, st>>>((double *)r->inc.p, (const float *)p->eps32.p,
                                                  (const PlaneWaveDev *)r->pw.p, ts, tsf, ph, Nx, Ny, Nz, t, nptr,
                                                  p->dt);
    } else
        k_incident<<<grid_for(nv * r->B), 256, 0, st>>>((double *)r->inc.p, (const double *)p->eps.p,
                                                              (const PlaneWaveDev *)r->pw.p, Nx, Ny, Nz, p->h, t, r->B,
                                                              nptr, p->dt);
    MOT_CHECK_LAUNCH();
    const int kmax = (int)std::min<long>(r->n, p->ell);
    if (hist_streaming(r)) {
        // streaming accumulation over the ring into the full-z spectrum (the
        // lags 2.. partial sum, then lag 1 onto it), then the inverse z FFT of
        // the Nz kept planes.  In the step graph the partial sum is the one the
        // previous step computed beside its solve, and this step's branch
        // computes the next one.
        Octant oc = {Mz, My, p->Kh[2], p->Kh[1], H};
        C *acc = (C *)r->hacc.p;
        const unsigned blocks = hist_blocks(r, 32);
        if (!nptr) {
            if (!p->capturing) p->kt.begin(st, MOT_K_HIST_SIDE);
            MOT_TRY(hist_side_host<T>(r, st, blocks, 256, 0));
            if (!p->capturing) p->kt.end(st);
            r->hpart_ok = false;  // the slots now serve this step, not the next one
        }
        if (!p->capturing) p->kt.begin(st, MOT_K_Z_HISTORY);
        count_launch();
        k_hist_acc<T><<<blocks, 256, 0, st>>>((const C *)r->ring.p, Lh_of<T>(p), nullptr, acc, Mz, My, H, oc, r->B,
                                              p->ell, r->n, 1, 1, nptr, 0, qslots<T>(r, kQBase));
        MOT_CHECK_LAUNCH();
        if (nptr) {
            // beside the solve: the next step's block pass (at a block start) and near accumulation
            MOT_CUDA_TRY(cudaEventRecord(r->hfork, st));
            MOT_CUDA_TRY(cudaStreamWaitEvent(r->hside, r->hfork, 0));
            const int bt = hist_side_threads();
            if (hist_spread()) {
                MOT_TRY(hist_block_pass<T>(r, r->hside, 0, 0, kHistRecent, 0, 0, nptr, 1));
                MOT_TRY(hist_block_pass<T>(r, r->hside, 0, 0, kHistOld, 0, 0, nptr, 1));
            } else
                MOT_TRY(hist_block_pass<T>(r, r->hside, 0, 0, kHistAll, 0, 0, nptr, 1));
            MOT_TRY(hist_near<T>(r, r->hside, 0, nptr, 1, hist_blocks(r, hist_side_per_sm_x2(), bt), bt,
                                 hist_side_mode()));
            MOT_CUDA_TRY(cudaEventRecord(r->hjoin, r->hside));
            r->hjoin_open = true;
        }
        const long zp = (long)My * H;
        if (col_r<T, +1>(acc, Bf, tz, (int)zp, Mz, Nz, r->B * 3, (long)Mz * zp, (long)Nz * zp, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_axis<T, +1>(acc, Bf, tz, H, Mz, Nz, r->B * 3, My, (long)Mz * zp, H, zp, (long)Nz * zp, H, zp, st)));
        if (!p->capturing) p->kt.end(st);
    } else {
        // ~100 KB of shared memory per CTA keeps two CTAs resident per SM
        int tw = sizeof(T) == 4 ? 8 : 4;
        while (tw > 1 && (size_t)(12 * Mz * tw + Mz) * sizeof(C) > 112 * 1024) tw /= 2;
        size_t smem = (size_t)(12 * Mz * tw + Mz) * sizeof(C);
        MOT_TRY(allow_smem<k_z_history2<T>>());
        Octant oc = {Mz, My, p->Kh[2], p->Kh[1], H};
        dim3 grid((H + tw - 1) / tw, (unsigned)(r->B * (My / 2 + 1)));
        if (!p->capturing) p->kt.begin(st, MOT_K_Z_HISTORY);
        count_launch();
        k_z_history2<T><<<grid, kZThreads, smem, st>>>((const C *)r->ring.p, Lh_of<T>(p), Bf, planp<T>(tz), twp<T>(tz), Nz, My,
                                                 H, tw, oc, r->B, p->ell, r->n, kmax, nptr);
        if (!p->capturing) p->kt.end(st);
        MOT_CHECK_LAUNCH();
    }
    EpiHistory e;
    e.inc = (const double *)r->inc.p;
    e.pol = nullptr;  // set below
    e.Jprev = (nptr || r->n > 0) ? (const double *)r->J.p : nullptr;  // J = 0 before the first step
    e.out = (double *)r->b.p;
    e.eps = (const double *)p->eps.p;
    e.plane_rows = (long)Nz * Ny;
    e.Nx = Nx;
    e.nvox = nv;
    e.pol = (const double *)((const char *)r->pw.p + r->B * sizeof(PlaneWaveDev));
    if (xy_smem_bytes<T>(p->Mh[0], My, H, Ny) <= kSmemMax) {
        if (!p->capturing) p->kt.begin(st, MOT_K_INV_HISTORY);
        MOT_TRY((launch_xy_inverse<T, EpiHistory>(Bf, r->B * 3 * Nz, Nx, Ny, Nz, H, tx, ty, e, st)));
        if (!p->capturing) p->kt.end(st);
    } else {
        if (!p->capturing) p->kt.begin(st, MOT_K_INV_HISTORY);
        if (col_r<T, +1>(Bf, A, ty, H, My, Ny, r->B * 3 * Nz, (long)My * H, (long)Ny * H, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_axis<T, +1>(Bf, A, ty, H, My, Ny, r->B * 3 * Nz, 1, (long)My * H, 0, H, (long)Ny * H, 0, H, st)));
        if (x_inverse_r<T, EpiHistory>(A, (long)r->B * 3 * Nz * Ny, Nx, Ny, Nz, tx, e, st)) MOT_CHECK_LAUNCH();
        else MOT_TRY((launch_x_inverse<T, EpiHistory>(A, (long)r->B * 3 * Nz * Ny, Nx, H, tx, e, st)));
        if (!p->capturing) p->kt.end(st);
    }
    return MOT_OK;
}

mot_status norms(mot_run *r, const double *v, double *out_host) {
    mot_problem *p = r->p;
    cudaStream_t st = p->ctx->stream;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    count_launch();
    k_norm2<<<dim3(kRedBlocks, r->B), kRedThreads, 0, st>>>(v, L, (double *)r->part1.p, (double *)r->dots.p,
                                                          (unsigned *)r->ctr.p + 3);
    MOT_CHECK_LAUNCH();
    MOT_CUDA_TRY(cudaMemcpyAsync(out_host, r->dots.p, sizeof(double) * r->B, cudaMemcpyDeviceToHost, st));
    MOT_CUDA_TRY(cudaStreamSynchronize(st));
    for (int b = 0; b < r->B; ++b) out_host[b] = sqrt(out_host[b]);
    return MOT_OK;
}

// one MOT step (Eq. 3)
mot_status run_one_step(mot_run *r, mot_step_stats *stats) {
    mot_problem *p = r->p;
    cudaStream_t st = p->ctx->stream;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    const long n = L * r->B;
    const long pr = (long)p->N[2] * p->N[1];
    const bool mixed = r->prec == MOT_MIXED, dfm = r->prec == MOT_FP64DF;
    p->kt.on = p->opt.timing != 0;
    p->kt.reset();
    int mvps = 0;
    cudaEventRecord(r->ev[0], st);
    if (mixed) MOT_TRY(history_rhs<float>(r, st));
    else if (dfm) MOT_TRY(history_rhs<dfl>(r, st));
    else MOT_TRY(history_rhs<double>(r, st));
    cudaEventRecord(r->ev[1], st);
    MOT_TRY(launch_guess(r, n, st));
    int iters = 0, sweeps = 0;
    bool conv = true;
    std::vector<double> bn(r->B), rn(r->B);
    MOT_TRY(norms(r, (const double *)r->b.p, bn.data()));
    double relres = 0.0;
    if (!mixed && !dfm) {
        const double tol = p->opt.tol > 0 ? p->opt.tol : 1e-11;
        int it;
        bool c;
        int nm;
        MOT_TRY(tfqmr<double>(r, (double *)r->J.p, (const double *)r->b.p, false, tol, p->opt.maxit, &it, &c, &nm));
        mvps += nm;
        iters = it;
        conv = c;
        sweeps = 1;
        EpiResidual e = {(const double *)r->J.p, (const double *)r->b.p, (double *)r->r.p, (const double *)p->eps.p, pr,
                         p->N[0], p->opt.delta};
        MOT_TRY((z0_product<double, double>(p, (const double *)r->J.p, r->B, p->wsA.p, p->wsB.p, e, st)));
        ++mvps;
        MOT_TRY(norms(r, (const double *)r->r.p, rn.data()));
    } else {
        const double tol = outer_tol(r);
        float *r32 = (float *)r->r32.p;
        float *c32 = r32 + n;
        MOT_TRY(dev_norms2(r, (const double *)r->b.p, (double *)r->b2.p, st));
        const InnerTol itol = inner_tol_for(r, (const double *)r->dots.p, tol);
        for (sweeps = 0; sweeps <= p->opt.max_refine; ++sweeps) {
            MOT_TRY(residual_product(r, st));
            ++mvps;
            MOT_TRY(norms(r, (const double *)r->r.p, rn.data()));
            bool done = true;
            for (int b = 0; b < r->B; ++b)
                if (rn[b] > tol * bn[b]) done = false;
            if (done || sweeps == p->opt.max_refine) break;
            // r->dots holds the squared residual norms (norms above)
            const dim3 gs(grid_for(L), r->B);
            int it;
            bool c;
            int nm;
            if (fused_start<float>(p)) {  // the start kernel scales and converts r itself
                MOT_TRY(tfqmr<float>(r, c32, nullptr, true, p->opt.inner_tol, p->opt.maxit, &it, &c, &nm,
                                     (const double *)r->r.p, (const double *)r->dots.p, itol));
            } else {
                count_launch();
                k_convert_scaled<<<gs, 256, 0, st>>>(r32, (const double *)r->r.p, (const double *)r->dots.p, L);
                MOT_CHECK_LAUNCH();
                MOT_TRY(tfqmr<float>(r, c32, r32, true, p->opt.inner_tol, p->opt.maxit, &it, &c, &nm, nullptr,
                                     nullptr, itol));
            }
            mvps += nm;
            iters += it;
            count_launch();
            k_add_scaled<<<gs, 256, 0, st>>>((double *)r->J.p, c32, (const double *)r->dots.p, L);
            MOT_CHECK_LAUNCH();
        }
        conv = true;
        for (int b = 0; b < r->B; ++b)
            if (rn[b] > tol * bn[b]) conv = false;
    }
    for (int b = 0; b < r->B; ++b) relres = std::max(relres, bn[b] > 0 ? rn[b] / bn[b] : 0.0);
    cudaEventRecord(r->ev[2], st);
    if (mixed) MOT_TRY(ring_push<float>(r, st));
    else if (dfm) MOT_TRY(ring_push<dfl>(r, st));
    else MOT_TRY(ring_push<double>(r, st));
    cudaEventRecord(r->ev[3], st);
    if (stats) {
        MOT_CUDA_TRY(cudaEventSynchronize(r->ev[3]));
        stats->iters = iters;
        stats->sweeps = sweeps;
        stats->relres = relres;
        cudaEventElapsedTime(&stats->ms_history, r->ev[0], r->ev[1]);
        cudaEventElapsedTime(&stats->ms_solve, r->ev[1], r->ev[2]);
        cudaEventElapsedTime(&stats->ms_push, r->ev[2], r->ev[3]);
        stats->mvps = (int32_t)mvps;
        stats->ms_zhist = p->kt.total(MOT_K_Z_HISTORY);
        const int ng = p->kt.count(MOT_K_Z_GREEN);
        stats->ms_zgreen = ng > 0 ? p->kt.total(MOT_K_Z_GREEN) / ng : 0.f;
    }
    p->kt.on = false;
    r->n += 1;
    if (!conv) {
        set_error("TFQMR did not reach the tolerance at step " + std::to_string(r->n - 1) +
                  " (relres " + std::to_string(relres) + ")");
        return MOT_ENOTCONV;
    }
    return MOT_OK;
}

// ============================================================================
// graph mode: one CUDA graph per MOT step, control kept on the device
// ============================================================================
struct StepDev {
    long long n;     // index of the step being computed
    int iters;       // TFQMR iterations of the step (sum over sweeps)
    int sweeps;      // refinement sweeps
    int mvps;        // Z0 products
    int notconv;     // 1 if the step missed its tolerance
    double relres;   // max_b ||b - Z0 J|| / ||b||
    int nstat;       // index of this step within the current mot_run_step call
    int loops;       // TFQMR loop-body executions of the step (sum over solves)
};

struct StepStatDev {
    int iters, sweeps, mvps, notconv;
    double relres;
    int loops, pad;
};

__global__ void k_step_begin(StepDev *s) {
    if (threadIdx.x == 0) {
        s->iters = 0;
        s->sweeps = 0;
        s->mvps = 0;
        s->notconv = 0;
        s->relres = 0.0;
        s->loops = 0;
    }
}

// start of an inner TFQMR loop: reset its iteration counter and condition
__global__ void k_cond_set(cudaGraphConditionalHandle h, int *ctl, int maxit) {
    if (threadIdx.x == 0) {
        ctl[0] = 0;
        ctl[1] = maxit;
        cudaGraphSetConditional(h, 1u);
    }
}

// after a solve: iterations, products, convergence into the step record
__global__ void k_solve_stats(const TfqmrScal *sc, int B, const int *ctl, StepDev *s, int init_mvps, int mark) {
    if (threadIdx.x == 0) {
        int mx = 0, bad = 0;
        for (int b = 0; b < B; ++b) {
            int it = (sc[b].m + 1) / 2;
            mx = it > mx ? it : mx;
            if (sc[b].conv == 0) bad = 1;
        }
        s->iters += mx;
        s->mvps += init_mvps + 2 * ctl[0];
        s->loops += ctl[0];
        if (mark && bad) s->notconv = 1;
    }
}

// refinement control: stop once every ||r_b|| <= tol ||b_b|| or after
// max_refine sweeps; counts the residual product that preceded it
__global__ void k_refine_cond(cudaGraphConditionalHandle h, const double *b2, const double *r2, int B, double tol,
                              int max_refine, StepDev *s, int after_sweep) {
    if (threadIdx.x == 0) {
        int done = 1;
        double rel = 0.0;
        for (int b = 0; b < B; ++b) {
            double bn = sqrt(b2[b]), rn = sqrt(r2[b]);
            if (rn > tol * bn) done = 0;
            double q = bn > 0.0 ? rn / bn : 0.0;
            rel = q > rel ? q : rel;
        }
        s->relres = rel;
        s->mvps += 1;
        if (after_sweep) s->sweeps += 1;
        int cont = (!done && s->sweeps < max_refine) ? 1 : 0;
        if (!done && !cont) s->notconv = 1;
        cudaGraphSetConditional(h, (unsigned)cont);
    }
}

// FP64 path: relative residual after the solve
__global__ void k_fp64_finish(const double *b2, const double *r2, int B, StepDev *s) {
    if (threadIdx.x == 0) {
        double rel = 0.0;
        for (int b = 0; b < B; ++b) {
            double bn = sqrt(b2[b]), rn = sqrt(r2[b]);
            double q = bn > 0.0 ? rn / bn : 0.0;
            rel = q > rel ? q : rel;
        }
        s->relres = rel;
        s->mvps += 1;
        s->sweeps = 1;
    }
}

__global__ void k_step_end(StepDev *s, StepStatDev *out, int cap) {
    if (threadIdx.x == 0) {
        int i = s->nstat;
        if (i >= 0 && i < cap) {
            StepStatDev d;
            d.iters = s->iters;
            d.sweeps = s->sweeps;
            d.mvps = s->mvps;
            d.notconv = s->notconv;
            d.relres = s->relres;
            d.loops = s->loops;
            d.pad = 0;
            out[i] = d;
        }
        s->nstat = i + 1;
        s->n += 1;
    }
}

// squared 2-norms of the batch vectors into out[B] (device only)
mot_status dev_norms2(mot_run *r, const double *v, double *out, cudaStream_t st) {
    mot_problem *p = r->p;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    count_launch();
    k_norm2<<<dim3(kRedBlocks, r->B), kRedThreads, 0, st>>>(v, L, (double *)r->part1.p, out, (unsigned *)r->ctr.p + 3);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

// conditional WHILE node inserted into the graph being captured on st; the
// body is captured on bst by fn(bst); work captured on st afterwards depends
// on the node.  The handle is created on `owner` before fn runs and is also
// returned so kernels captured before the node can set it.
struct WhileNode {
    cudaGraphConditionalHandle h;
    cudaGraph_t owner;
};

mot_status while_handle(cudaStream_t st, WhileNode &w, unsigned defv) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    MOT_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive || !g) MOT_FAIL(MOT_ECUDA, "stream is not capturing");
    MOT_CUDA_TRY(cudaGraphConditionalHandleCreate(&w.h, g, defv, cudaGraphCondAssignDefault));
    w.owner = g;
    return MOT_OK;
}

template <class F>
mot_status while_insert(cudaStream_t st, cudaStream_t bst, const WhileNode &w, F fn, int *body_kernels = nullptr) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    MOT_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = w.h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    MOT_CUDA_TRY(cudaGraphAddNode(&node, g, dv.data(), nullptr, nd, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MOT_CUDA_TRY(cudaStreamBeginCaptureToGraph(bst, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const unsigned long long b0 = g_launches.load();
    mot_status s = fn(bst);
    if (body_kernels) *body_kernels = (int)(g_launches.load() - b0);
    cudaGraph_t tmp = nullptr;
    cudaError_t ce = cudaStreamEndCapture(bst, &tmp);
    if (s != MOT_OK) return s;
    if (ce != cudaSuccess) MOT_FAIL(MOT_ECUDA, std::string("body capture: ") + cudaGetErrorString(ce));
    MOT_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return MOT_OK;
}

// TFQMR solve captured on st (start kernels, WHILE node with the iteration
// body captured on bst, flush), solve statistics into the step record
template <typename V>
mot_status tfqmr_capture(mot_run *r, V *x, const V *rhs, bool zero_x0, double tol, int maxit, cudaStream_t st,
                         cudaStream_t bst, int mark_notconv, const double *src64 = nullptr,
                         const double *n2 = nullptr, InnerTol itol = InnerTol{}) {
    mot_problem *p = r->p;
    const int B = r->B;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    KrylovView<V> k = kview<V>(r);
    dim3 gv(grid_for(L), B);
    int init_mvps = 1;
    MOT_TRY(tfqmr_start<V>(r, x, rhs, zero_x0, tol, st, &init_mvps, src64, n2, itol));
    WhileNode w;
    MOT_TRY(while_handle(st, w, 1));
    count_launch();
    k_cond_set<<<1, 32, 0, st>>>(w.h, (int *)r->ctl.p, maxit);
    MOT_CHECK_LAUNCH();
    MOT_TRY(while_insert(st, bst, w, [&](cudaStream_t cs) -> mot_status {
        return tfqmr_body<V>(r, x, cs, w.h, 1);
    }, &r->k_inner));
    count_launch();
    k_tfqmr_flush<V, V><<<gv, 256, 0, st>>>(x, k.v[kD], k.sc, L, 1);
    count_launch();
    k_solve_stats<<<1, 32, 0, st>>>(k.sc, B, (const int *)r->ctl.p, (StepDev *)r->sdev.p, init_mvps, mark_notconv);
    count_launch();
    k_tfqmr_settle<<<(B + 255) / 256, 256, 0, st>>>(k.sc, B, 1);
    MOT_CHECK_LAUNCH();
    return MOT_OK;
}

// capture one whole MOT step (Eq. 3) into r->step_graph
mot_status build_step_graph(mot_run *r) {
    mot_problem *p = r->p;
    const bool mixed = r->prec == MOT_MIXED, dfm = r->prec == MOT_FP64DF;
    const long L = 3L * p->N[0] * p->N[1] * p->N[2];
    const long n = L * r->B;
    const long pr = (long)p->N[2] * p->N[1];
    StepDev *sd = (StepDev *)r->sdev.p;
    const long long *nptr = (const long long *)r->sdev.p;  // StepDev::n is the first member
    cudaStream_t st = r->cap;
    p->capturing = true;
    const unsigned long long l0 = g_launches.load();
    MOT_CUDA_TRY(cudaGraphCreate(&r->step_graph, 0));
    MOT_CUDA_TRY(cudaStreamBeginCaptureToGraph(st, r->step_graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    auto body = [&]() -> mot_status {
        count_launch();
        k_step_begin<<<1, 32, 0, st>>>(sd);
        MOT_CHECK_LAUNCH();
        if (mixed) MOT_TRY(history_rhs<float>(r, st, nptr));
        else if (dfm) MOT_TRY(history_rhs<dfl>(r, st, nptr));
        else MOT_TRY(history_rhs<double>(r, st, nptr));
        MOT_TRY(launch_guess(r, n, st));
        MOT_TRY(dev_norms2(r, (const double *)r->b.p, (double *)r->b2.p, st));
        if (!mixed && !dfm) {
            const double tol = p->opt.tol > 0 ? p->opt.tol : 1e-11;
            MOT_TRY(tfqmr_capture<double>(r, (double *)r->J.p, (const double *)r->b.p, false, tol, p->opt.maxit, st,
                                          r->cap2, 1));
            EpiResidual e = {(const double *)r->J.p, (const double *)r->b.p, (double *)r->r.p,
                             (const double *)p->eps.p, pr, p->N[0], p->opt.delta};
            MOT_TRY((z0_product<double, double>(p, (const double *)r->J.p, r->B, p->wsA.p, p->wsB.p, e, st)));
            MOT_TRY(dev_norms2(r, (const double *)r->r.p, (double *)r->r2.p, st));
            count_launch();
            k_fp64_finish<<<1, 32, 0, st>>>((const double *)r->b2.p, (const double *)r->r2.p, r->B, sd);
            MOT_CHECK_LAUNCH();
            MOT_TRY(ring_push<double>(r, st, nptr));
        } else {
            const double tol = outer_tol(r);
            float *r32 = (float *)r->r32.p;
            float *c32 = r32 + n;
            // residual of the initial guess, then sweeps while it misses tol
            MOT_TRY(residual_product(r, st));
            MOT_TRY(dev_norms2(r, (const double *)r->r.p, (double *)r->r2.p, st));
            WhileNode wo;
            MOT_TRY(while_handle(st, wo, 0));
            count_launch();
            k_refine_cond<<<1, 32, 0, st>>>(wo.h, (const double *)r->b2.p, (const double *)r->r2.p, r->B, tol,
                                            p->opt.max_refine, sd, 0);
            MOT_CHECK_LAUNCH();
            MOT_TRY(while_insert(st, r->cap2, wo, [&](cudaStream_t cs) -> mot_status {
                // r->r2 holds the squared residual norms (dev_norms2 before the test)
                const dim3 gs(grid_for(L), r->B);
                const InnerTol itol = inner_tol_for(r, (const double *)r->r2.p, tol);
                if (fused_start<float>(p)) {  // the start kernel scales and converts r itself
                    MOT_TRY(tfqmr_capture<float>(r, c32, nullptr, true, p->opt.inner_tol, p->opt.maxit, cs, r->cap3,
                                                 0, (const double *)r->r.p, (const double *)r->r2.p, itol));
                } else {
                    count_launch();
                    k_convert_scaled<<<gs, 256, 0, cs>>>(r32, (const double *)r->r.p, (const double *)r->r2.p, L);
                    MOT_CHECK_LAUNCH();
                    MOT_TRY(tfqmr_capture<float>(r, c32, r32, true, p->opt.inner_tol, p->opt.maxit, cs, r->cap3, 0,
                                                 nullptr, nullptr, itol));
                }
                count_launch();
                k_add_scaled<<<gs, 256, 0, cs>>>((double *)r->J.p, c32, (const double *)r->r2.p, L);
                MOT_CHECK_LAUNCH();
                MOT_TRY(residual_product(r, cs));
                MOT_TRY(dev_norms2(r, (const double *)r->r.p, (double *)r->r2.p, cs));
                count_launch();
                k_refine_cond<<<1, 32, 0, cs>>>(wo.h, (const double *)r->b2.p, (const double *)r->r2.p, r->B, tol,
                                                p->opt.max_refine, sd, 1);
                MOT_CHECK_LAUNCH();
                return MOT_OK;
            }, &r->k_outer));
            r->k_outer -= r->k_inner;  // the nested loop body is counted per iteration
            if (dfm) MOT_TRY(ring_push<dfl>(r, st, nptr));
            else MOT_TRY(ring_push<float>(r, st, nptr));
        }
        if (r->hjoin_open) {  // the next step's partial history sum is part of this step
            MOT_CUDA_TRY(cudaStreamWaitEvent(st, r->hjoin, 0));
            r->hjoin_open = false;
        }
        count_launch();
        k_step_end<<<1, 32, 0, st>>>(sd, (StepStatDev *)r->sstats.p, r->sstats_cap);
        MOT_CHECK_LAUNCH();
        return MOT_OK;
    };
    r->k_outer = 0;
    r->k_inner = 0;
    mot_status s = body();
    cudaGraph_t out = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &out);
    p->capturing = false;
    const unsigned long long captured = g_launches.load() - l0;
    g_launches.fetch_sub(captured);  // captured, not launched: counted per executed step
    r->k_fixed = (int)captured - r->k_outer - r->k_inner;
    if (s != MOT_OK) return s;
    if (ce != cudaSuccess) MOT_FAIL(MOT_ECUDA, std::string("step capture: ") + cudaGetErrorString(ce));
    // node priorities: the captured nodes keep their streams' priorities (the solve's
    // and the side branch's streams are both at the highest)
    cudaError_t ie = cudaGraphInstantiate(&r->step_exec, r->step_graph, cudaGraphInstantiateFlagUseNodePriority);
    if (ie != cudaSuccess) {
        cudaGetLastError();
        ie = cudaGraphInstantiate(&r->step_exec, r->step_graph, 0);
    }
    if (ie != cudaSuccess) MOT_FAIL(MOT_ECUDA, std::string("step graph instantiate: ") + cudaGetErrorString(ie));
    return MOT_OK;
}

}  // namespace

extern "C" {

mot_status mot_run_create(mot_problem *p, int nrhs, const mot_planewave *exc, int precision, mot_run **out) {
    if (!p || !exc || !out) MOT_FAIL(MOT_EINVAL, "NULL argument");
    *out = nullptr;
    if (nrhs < 1 || nrhs > 1024) MOT_FAIL(MOT_EINVAL, "nrhs out of range [1, 1024]");
    if (precision != MOT_FP64 && precision != MOT_MIXED && precision != MOT_FP64DF)
        MOT_FAIL(MOT_EINVAL, "precision must be MOT_FP64, MOT_MIXED or MOT_FP64DF");
    for (int b = 0; b < nrhs; ++b) {
        const mot_planewave &w = exc[b];
        double kk = 0, pp = 0, kp = 0;
        for (int i = 0; i < 3; ++i) {
            kk += w.khat[i] * w.khat[i];
            pp += w.pol[i] * w.pol[i];
            kp += w.khat[i] * w.pol[i];
        }
        if (fabs(kk - 1.0) > 1e-9 || fabs(pp - 1.0) > 1e-9 || fabs(kp) > 1e-9)
            MOT_FAIL(MOT_EINVAL, "plane wave: khat and pol must be orthogonal unit vectors");
        if (!(w.sigma > 0.0) || !std::isfinite(w.E0) || !std::isfinite(w.t0) || !std::isfinite(w.f0) ||
            !std::isfinite(w.sigma))
            MOT_FAIL(MOT_EINVAL, "plane wave: sigma must be > 0 and all parameters finite");
    }
    MOT_CUDA_TRY(cudaSetDevice(p->ctx->device));
    PhaseTrace tr_run("run creation");
    const bool mixed = precision == MOT_MIXED;
    const bool inner32 = precision != MOT_FP64;  // FP32 inner solves refined against an outer residual
    MOT_TRY(build_history_spectra(p, mixed ? kSpec32 : precision == MOT_FP64DF ? kSpecDF : kSpec64));
    mot_run *r = new mot_run();
    r->p = p;
    r->B = nrhs;
    r->prec = precision;
    auto fail = [&](mot_status s) {
        mot_run_destroy(r);
        return s;
    };
    const long nv = (long)p->N[0] * p->N[1] * p->N[2];
    const long n = 3 * nv * nrhs;
    r->exc_host.assign(exc, exc + nrhs);
    // plane waves, then pol[B][3] right after them
    r->pw_host.resize(nrhs);
    std::vector<double> pol(3 * nrhs);
    for (int b = 0; b < nrhs; ++b) {
        PlaneWaveDev d;
        d.E0 = exc[b].E0;
        d.sigma = exc[b].sigma;
        d.t0 = exc[b].t0;
        d.f0 = exc[b].f0;
        for (int i = 0; i < 3; ++i) {
            d.khat[i] = exc[b].khat[i];
            d.pol[i] = exc[b].pol[i];
            d.rref[i] = exc[b].khat[i] < 0 ? p->N[i] * p->h : 0.0;
            pol[3 * b + i] = exc[b].pol[i];
        }
        planewave_factors(d, p->h);
        r->pw_host[b] = d;
    }
    mot_status s;
    {
        // axis tables of the fast incident path: ts[B][S] doubles, ph[B][S] float2, tsf[B][S] floats
        const long S = (long)p->N[0] + p->N[1] + p->N[2];
        std::vector<double> ts(S * nrhs);
        std::vector<float2> ph(S * nrhs);
        std::vector<float> tsf(S * nrhs);
        for (int b = 0; b < nrhs; ++b)
            incident_tables(r->pw_host[b], p->N, p->h, ts.data() + b * S, tsf.data() + b * S, ph.data() + b * S);
        if ((s = dalloc(r->inctab, (sizeof(double) + sizeof(float2) + sizeof(float)) * S * nrhs)) != MOT_OK)
            return fail(s);
        char *base = (char *)r->inctab.p;
        if (cudaMemcpy(base, ts.data(), sizeof(double) * S * nrhs, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(base + sizeof(double) * S * nrhs, ph.data(), sizeof(float2) * S * nrhs,
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(base + (sizeof(double) + sizeof(float2)) * S * nrhs, tsf.data(), sizeof(float) * S * nrhs,
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(MOT_ECUDA);
    }
    if ((s = dalloc(r->pw, sizeof(PlaneWaveDev) * nrhs + sizeof(double) * 3 * nrhs)) != MOT_OK) return fail(s);
    cudaMemcpy(r->pw.p, r->pw_host.data(), sizeof(PlaneWaveDev) * nrhs, cudaMemcpyHostToDevice);
    cudaMemcpy((char *)r->pw.p + sizeof(PlaneWaveDev) * nrhs, pol.data(), sizeof(double) * 3 * nrhs,
               cudaMemcpyHostToDevice);
    const size_t cs = mixed ? sizeof(float2) : sizeof(double2);  // history element (dfl2: 16 bytes too)
    const size_t vs = inner32 ? sizeof(float) : sizeof(double);   // Krylov vectors
    if ((s = dalloc(r->inc, sizeof(double) * nv * nrhs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->J, sizeof(double) * n)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->J2, sizeof(double) * n)) != MOT_OK) return fail(s);
    if (p->opt.guess == 2 && (s = dalloc(r->J3, sizeof(double) * n)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->b, sizeof(double) * n)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->r, sizeof(double) * n)) != MOT_OK) return fail(s);
    size_t ring_bytes = (size_t)p->ell * nrhs * 3 * p->Mh[2] * p->Mh[1] * p->Hh * cs;
    if ((s = dalloc(r->ring, ring_bytes)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->hacc, ring_bytes / p->ell)) != MOT_OK) return fail(s);
    // time block: 8 steps in FP32, 4 in FP64 and double-float (the block pass holds that many outputs in registers)
    r->hTB = mixed ? 8 : 4;
    if ((s = dalloc(r->hpart, ring_bytes / p->ell * (2 * r->hTB))) != MOT_OK) return fail(s);
    if ((s = dalloc(r->wsAh, (size_t)nrhs * 3 * p->N[2] * p->N[1] * p->Hh * cs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->wsBh, (size_t)nrhs * 3 * p->N[2] * p->Mh[1] * p->Hh * cs)) != MOT_OK) return fail(s);
    for (int i = 0; i < 10; ++i)
        if ((s = dalloc(r->kv[i], vs * n)) != MOT_OK) return fail(s);
    if (inner32 && (s = dalloc(r->r32, sizeof(float) * 2 * n)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->scal, sizeof(TfqmrScal) * nrhs)) != MOT_OK) return fail(s);
    // partial sums per right-hand side: kRedBlocks blocks or one per (component, z) plane
    const long nparts = std::max<long>(kRedBlocks, 3L * p->N[2]);
    if ((s = dalloc(r->part1, sizeof(double) * nparts * nrhs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->part2, sizeof(double) * nparts * nrhs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->part3, sizeof(double) * nparts * nrhs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->dots, sizeof(double) * nrhs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->ctl, sizeof(int) * 4)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->ctr, sizeof(unsigned) * 4)) != MOT_OK) return fail(s);
    if (cudaMemset(r->ctr.p, 0, sizeof(unsigned) * 4) != cudaSuccess) return fail(MOT_ECUDA);
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) return fail(MOT_ECUDA);
    if (cudaStreamCreateWithPriority(&r->cap, cudaStreamNonBlocking, prio_hi) != cudaSuccess) return fail(MOT_ECUDA);
    if (cudaStreamCreateWithPriority(&r->cap2, cudaStreamNonBlocking, prio_hi) != cudaSuccess) return fail(MOT_ECUDA);
    if (cudaStreamCreateWithPriority(&r->cap3, cudaStreamNonBlocking, prio_hi) != cudaSuccess) return fail(MOT_ECUDA);
    // the history side branch at the solve's priority: the time-blocked pass shares the SMs
    // with the solve's kernels instead of filling their gaps only (256x256x80: 92.6 against
    // 87.8 steps/s at the lowest priority; 64^3 alike either way)
    if (cudaStreamCreateWithPriority(&r->hside, cudaStreamNonBlocking, prio_hi) != cudaSuccess) return fail(MOT_ECUDA);
    if (cudaEventCreateWithFlags(&r->hfork, cudaEventDisableTiming) != cudaSuccess) return fail(MOT_ECUDA);
    if (cudaEventCreateWithFlags(&r->hjoin, cudaEventDisableTiming) != cudaSuccess) return fail(MOT_ECUDA);
    r->sstats_cap = 1024;
    if ((s = dalloc(r->sdev, sizeof(StepDev))) != MOT_OK) return fail(s);
    if ((s = dalloc(r->sstats, sizeof(StepStatDev) * r->sstats_cap)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->b2, sizeof(double) * nrhs)) != MOT_OK) return fail(s);
    if ((s = dalloc(r->r2, sizeof(double) * nrhs)) != MOT_OK) return fail(s);
    cudaMemsetAsync(r->sdev.p, 0, sizeof(StepDev), p->ctx->stream);

    // Z0 workspace for the batch in both precisions (FP64 residual / FP32 inner)
    size_t a, bb;
    z0_ws_bytes(p, nrhs, sizeof(double2), &a, &bb);
    if ((s = dalloc(p->wsA, a)) != MOT_OK) return fail(s);
    if ((s = dalloc(p->wsB, bb)) != MOT_OK) return fail(s);
    cudaStream_t st = p->ctx->stream;
    cudaMemsetAsync(r->ring.p, 0, ring_bytes, st);
    cudaMemsetAsync(r->hpart.p, 0, r->hpart.bytes, st);
    cudaMemsetAsync(r->J.p, 0, sizeof(double) * n, st);
    cudaMemsetAsync(r->J2.p, 0, sizeof(double) * n, st);
    if (r->J3.p) cudaMemsetAsync(r->J3.p, 0, sizeof(double) * n, st);
    for (int i = 0; i < 4; ++i)
        if (cudaEventCreate(&r->ev[i]) != cudaSuccess) return fail(MOT_ECUDA);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(MOT_ECUDA);
    {   // launch schedule of the batch's products (tuned once per problem and precision)
        const Sched *sc = nullptr;
        s = inner32 ? schedule_for<float>(p, nrhs, &sc) : schedule_for<double>(p, nrhs, &sc);
        if (s != MOT_OK) return fail(s);
    }
    *out = r;
    return MOT_OK;
}

// the staging buffers, copy stream and events of the overlapped J_n copies
mot_status jcopy_setup(mot_run *r, long n) {
    for (int b = 0; b < 2; ++b) {
        if (!r->jstage[b].p) MOT_TRY(dalloc(r->jstage[b], sizeof(double) * n));
        if (!r->jready[b]) MOT_CUDA_TRY(cudaEventCreateWithFlags(&r->jready[b], cudaEventDisableTiming));
        if (!r->jdone[b]) MOT_CUDA_TRY(cudaEventCreateWithFlags(&r->jdone[b], cudaEventDisableTiming));
    }
    if (!r->jcopy) MOT_CUDA_TRY(cudaStreamCreateWithFlags(&r->jcopy, cudaStreamNonBlocking));
    return MOT_OK;
}

mot_status mot_run_step(mot_run *r, int nsteps, double *J_out, mot_step_stats *stats) {
    if (!r) MOT_FAIL(MOT_EINVAL, "run is NULL");
    if (nsteps < 0) MOT_FAIL(MOT_EINVAL, "nsteps < 0");
    MOT_CUDA_TRY(cudaSetDevice(r->p->ctx->device));
    SchedScope scope(r->p->sched_for(r->B, r->prec != MOT_FP64));
    const long n = 3L * r->p->N[0] * r->p->N[1] * r->p->N[2] * r->B;
    mot_status result = MOT_OK;
    // graph mode (default): after one eager step (which sets every kernel's
    // attributes), each step is one graph launch with its control on the
    // device; graph = 0 or 2 keeps host-driven steps
    const bool eager_env = r->p->opt.graph != 1;
    if (!eager_env && r->warmed && nsteps > 0) {
        cudaStream_t st = r->p->ctx->stream;
        if (!r->step_exec) MOT_TRY(build_step_graph(r));
        // device step index follows the host's
        long long n0 = r->n;
        MOT_CUDA_TRY(cudaMemcpyAsync(r->sdev.p, &n0, sizeof(long long), cudaMemcpyHostToDevice, st));
        MOT_TRY(hist_prime(r, st));
        int done = 0;
        while (done < nsteps) {
            const int chunk = std::min(nsteps - done, r->sstats_cap);
            MOT_CUDA_TRY(cudaMemsetAsync((char *)r->sdev.p + offsetof(StepDev, nstat), 0, sizeof(int), st));
            // per-step events are read once the chunk is done: no host wait between steps
            while (stats && (int)r->sev.size() < 2 * chunk) {
                cudaEvent_t e;
                MOT_CUDA_TRY(cudaEventCreate(&e));
                r->sev.push_back(e);
            }
            if (J_out) MOT_TRY(jcopy_setup(r, n));
            for (int i = 0; i < chunk; ++i) {
                const int sidx = done + i;
                if (stats) MOT_CUDA_TRY(cudaEventRecord(r->sev[2 * i], st));
                MOT_CUDA_TRY(cudaGraphLaunch(r->step_exec, st));
                r->n += 1;
                if (stats) MOT_CUDA_TRY(cudaEventRecord(r->sev[2 * i + 1], st));
                if (J_out) {
                    // J_n to a staging buffer (free once its previous host copy is done), then
                    // to the host on the copy stream while the next step runs
                    const int b = sidx & 1;
                    if (sidx >= 2) MOT_CUDA_TRY(cudaStreamWaitEvent(st, r->jdone[b], 0));
                    MOT_CUDA_TRY(cudaMemcpyAsync(r->jstage[b].p, r->J.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
                    MOT_CUDA_TRY(cudaEventRecord(r->jready[b], st));
                    MOT_CUDA_TRY(cudaStreamWaitEvent(r->jcopy, r->jready[b], 0));
                    MOT_CUDA_TRY(cudaMemcpyAsync(J_out + (size_t)sidx * n, r->jstage[b].p, sizeof(double) * n,
                                                 cudaMemcpyDeviceToHost, r->jcopy));
                    MOT_CUDA_TRY(cudaEventRecord(r->jdone[b], r->jcopy));
                }
            }
            std::vector<StepStatDev> hs(chunk);
            MOT_CUDA_TRY(cudaMemcpyAsync(hs.data(), r->sstats.p, sizeof(StepStatDev) * chunk, cudaMemcpyDeviceToHost, st));
            MOT_CUDA_TRY(cudaStreamSynchronize(st));
            if (J_out) MOT_CUDA_TRY(cudaStreamSynchronize(r->jcopy));
            for (int i = 0; stats && i < chunk; ++i) {
                mot_step_stats &S = stats[done + i];
                memset(&S, 0, sizeof(S));
                if (cudaEventElapsedTime(&S.ms_solve, r->sev[2 * i], r->sev[2 * i + 1]) != cudaSuccess) {
                    S.ms_solve = 0.f;
                    cudaGetLastError();
                }
            }
            for (int i = 0; i < chunk; ++i) {
                // kernels the step graph executed: fixed part, each refinement
                // sweep's body, each TFQMR loop iteration
                g_launches.fetch_add((unsigned long long)(r->k_fixed + r->k_outer * hs[i].sweeps +
                                                          r->k_inner * hs[i].loops));
                if (hs[i].notconv) {
                    result = MOT_ENOTCONV;
                    set_error("tolerance not reached at step " + std::to_string(r->n - chunk + i) + " (relres " +
                              std::to_string(hs[i].relres) + ")");
                }
                if (stats) {
                    mot_step_stats &S = stats[done + i];
                    S.iters = hs[i].iters;
                    S.sweeps = hs[i].sweeps;
                    S.relres = hs[i].relres;
                    S.mvps = hs[i].mvps;
                }
            }
            done += chunk;
        }
        return result;
    }
    for (int s = 0; s < nsteps; ++s) {
        if (!eager_env && r->warmed) {  // switch to graph mode after the first step
            mot_status g = mot_run_step(r, nsteps - s, J_out ? J_out + (size_t)s * n : nullptr, stats ? stats + s : nullptr);
            return g != MOT_OK ? g : result;
        }
        mot_status st = run_one_step(r, stats ? stats + s : nullptr);
        if (st != MOT_OK && st != MOT_ENOTCONV) return st;
        r->warmed = true;
        if (st == MOT_ENOTCONV) result = st;
        if (J_out) {
            MOT_CUDA_TRY(cudaMemcpyAsync(J_out + (size_t)s * n, r->J.p, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                         r->p->ctx->stream));
        }
    }
    if (J_out || stats) MOT_CUDA_TRY(cudaStreamSynchronize(r->p->ctx->stream));
    return result;
}

// ---------------------------------------------------------------- checkpoints
namespace {
struct CkptHeader {
    char magic[8];  // "MOTJVIE\0"
    uint32_t version;
    int32_t precision;
    int32_t N[3];
    int32_t nrhs;
    double h, alpha;
    int64_t n;  // next step index
    int32_t ell, pad;
    uint64_t eps_hash;    // FNV-1a over the eps_r bytes
    uint64_t vec_bytes;   // one [nrhs][3][n] FP64 array
    uint64_t ring_bytes;  // the whole history ring
    mot_options opt;
};
constexpr uint32_t kCkptVersion = 2;  // 2: mot_options gained autotune

uint64_t fnv1a(const void *data, size_t bytes) {
    const unsigned char *c = (const unsigned char *)data;
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < bytes; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

size_t run_ring_bytes(const mot_run *r) {
    const mot_problem *p = r->p;
    const size_t cs = r->prec == MOT_MIXED ? sizeof(float2) : sizeof(double2);
    return (size_t)p->ell * r->B * 3 * p->Mh[2] * p->Mh[1] * p->Hh * cs;
}

// device <-> file through a bounded host buffer
mot_status dev_to_file(FILE *f, const void *dev, size_t bytes) {
    std::vector<char> buf(std::min<size_t>(bytes, (size_t)64 << 20));
    for (size_t o = 0; o < bytes; o += buf.size()) {
        const size_t k = std::min(buf.size(), bytes - o);
        MOT_CUDA_TRY(cudaMemcpy(buf.data(), (const char *)dev + o, k, cudaMemcpyDeviceToHost));
        if (fwrite(buf.data(), 1, k, f) != k) MOT_FAIL(MOT_EINVAL, "checkpoint write failed");
    }
    return MOT_OK;
}

mot_status file_to_dev(FILE *f, void *dev, size_t bytes) {
    std::vector<char> buf(std::min<size_t>(bytes, (size_t)64 << 20));
    for (size_t o = 0; o < bytes; o += buf.size()) {
        const size_t k = std::min(buf.size(), bytes - o);
        if (fread(buf.data(), 1, k, f) != k) MOT_FAIL(MOT_EINVAL, "checkpoint truncated");
        MOT_CUDA_TRY(cudaMemcpy((char *)dev + o, buf.data(), k, cudaMemcpyHostToDevice));
    }
    return MOT_OK;
}

struct FileCloser {
    FILE *f;
    ~FileCloser() {
        if (f) fclose(f);
    }
};
}  // namespace

mot_status mot_run_save(mot_run *r, const char *path) {
    if (!r || !path) MOT_FAIL(MOT_EINVAL, "NULL argument");
    mot_problem *p = r->p;
    MOT_CUDA_TRY(cudaSetDevice(p->ctx->device));
    MOT_CUDA_TRY(cudaStreamSynchronize(p->ctx->stream));
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "MOTJVIE", 8);
    hd.version = kCkptVersion;
    hd.precision = r->prec;
    for (int i = 0; i < 3; ++i) hd.N[i] = p->N[i];
    hd.nrhs = r->B;
    hd.h = p->h;
    hd.alpha = p->alpha;
    hd.n = r->n;
    hd.ell = p->ell;
    hd.eps_hash = fnv1a(p->eps_host.data(), p->eps_host.size() * sizeof(double));
    hd.vec_bytes = sizeof(double) * 3 * (size_t)p->N[0] * p->N[1] * p->N[2] * r->B;
    hd.ring_bytes = run_ring_bytes(r);
    hd.opt = p->opt;
    FileCloser fc{fopen(path, "wb")};
    if (!fc.f) MOT_FAIL(MOT_EINVAL, std::string("cannot open checkpoint for writing: ") + path);
    if (fwrite(&hd, sizeof(hd), 1, fc.f) != 1 ||
        fwrite(r->exc_host.data(), sizeof(mot_planewave), r->B, fc.f) != (size_t)r->B)
        MOT_FAIL(MOT_EINVAL, "checkpoint write failed");
    MOT_TRY(dev_to_file(fc.f, r->J.p, hd.vec_bytes));
    MOT_TRY(dev_to_file(fc.f, r->J2.p, hd.vec_bytes));
    if (r->J3.p) MOT_TRY(dev_to_file(fc.f, r->J3.p, hd.vec_bytes));  // guess 2 (hd.opt.guess says so)
    MOT_TRY(dev_to_file(fc.f, r->ring.p, hd.ring_bytes));
    if (fflush(fc.f) != 0) MOT_FAIL(MOT_EINVAL, "checkpoint write failed");
    return MOT_OK;
}

mot_status mot_run_load(mot_problem *p, const char *path, mot_run **out) {
    if (!p || !path || !out) MOT_FAIL(MOT_EINVAL, "NULL argument");
    *out = nullptr;
    FileCloser fc{fopen(path, "rb")};
    if (!fc.f) MOT_FAIL(MOT_EINVAL, std::string("cannot open checkpoint: ") + path);
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, fc.f) != 1 || memcmp(hd.magic, "MOTJVIE", 8) != 0)
        MOT_FAIL(MOT_EINVAL, "not a libmotjvie checkpoint");
    if (hd.version != kCkptVersion) MOT_FAIL(MOT_EINVAL, "checkpoint version not supported");
    bool same = hd.h == p->h && hd.alpha == p->alpha && hd.ell == p->ell &&
                hd.eps_hash == fnv1a(p->eps_host.data(), p->eps_host.size() * sizeof(double));
    for (int i = 0; i < 3; ++i) same = same && hd.N[i] == p->N[i];
    if (!same) MOT_FAIL(MOT_EINVAL, "checkpoint belongs to another problem (grid, h, alpha or eps_r differ)");
    if (hd.nrhs < 1 || hd.nrhs > 1024 || hd.n < 0) MOT_FAIL(MOT_EINVAL, "corrupt checkpoint header");
    std::vector<mot_planewave> exc(hd.nrhs);
    if (fread(exc.data(), sizeof(mot_planewave), hd.nrhs, fc.f) != (size_t)hd.nrhs)
        MOT_FAIL(MOT_EINVAL, "checkpoint truncated");
    mot_run *r = nullptr;
    MOT_TRY(mot_run_create(p, hd.nrhs, exc.data(), hd.precision, &r));
    const size_t vec = sizeof(double) * 3 * (size_t)p->N[0] * p->N[1] * p->N[2] * r->B;
    mot_status s = MOT_OK;
    if (hd.vec_bytes != vec || hd.ring_bytes != run_ring_bytes(r)) {
        set_error("checkpoint sizes do not match the run it describes");
        s = MOT_EINVAL;
    }
    if (s == MOT_OK) s = file_to_dev(fc.f, r->J.p, vec);
    if (s == MOT_OK) s = file_to_dev(fc.f, r->J2.p, vec);
    // J_{n-3}: stored when the saving run used guess 2; a run that needs it but finds
    // none takes J_{n-2} in its place (one less accurate first guess), one that does
    // not need it skips it
    if (s == MOT_OK && hd.opt.guess == 2) {
        if (r->J3.p) s = file_to_dev(fc.f, r->J3.p, vec);
        else if (fseek(fc.f, (long)vec, SEEK_CUR) != 0) {
            set_error("checkpoint truncated");
            s = MOT_EINVAL;
        }
    } else if (s == MOT_OK && r->J3.p) {
        if (cudaMemcpy(r->J3.p, r->J2.p, vec, cudaMemcpyDeviceToDevice) != cudaSuccess) {
            set_error("cudaMemcpy of J_{n-2} into J_{n-3} failed");
            s = MOT_ECUDA;
        }
    }
    if (s == MOT_OK) s = file_to_dev(fc.f, r->ring.p, hd.ring_bytes);
    if (s != MOT_OK) {
        mot_run_destroy(r);
        return s;
    }
    r->n = hd.n;
    r->q_stale = true;  // the time-block slots are rebuilt from the ring before the next step
    r->hpart_ok = false;
    *out = r;
    return MOT_OK;
}

mot_status mot_run_kernel_times(mot_run *r, int cls, int32_t *launches, float *mean_ms) {
    if (!r || !launches || !mean_ms) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (cls < 0 || cls >= MOT_K_CLASSES) MOT_FAIL(MOT_EINVAL, "kernel class out of range");
    MOT_CUDA_TRY(cudaSetDevice(r->p->ctx->device));
    MOT_CUDA_TRY(cudaStreamSynchronize(r->p->ctx->stream));
    const int n = r->p->kt.count(cls);
    *launches = n;
    *mean_ms = n > 0 ? r->p->kt.total(cls) / n : 0.f;
    return MOT_OK;
}

mot_status mot_run_current_device(mot_run *r, const void **J_dev) {
    if (!r || !J_dev) MOT_FAIL(MOT_EINVAL, "NULL argument");
    *J_dev = r->J.p;
    return MOT_OK;
}

mot_status mot_kernel_launches(uint64_t *count) {
    if (!count) MOT_FAIL(MOT_EINVAL, "count is NULL");
    *count = g_launches.load();
    return MOT_OK;
}

mot_status mot_fma_peak(int device, int dtype, double *flop_per_s, double *ms) {
    if (!flop_per_s) MOT_FAIL(MOT_EINVAL, "flop_per_s is NULL");
    if (dtype != MOT_F64 && dtype != MOT_F32) MOT_FAIL(MOT_EINVAL, "dtype must be MOT_F64 or MOT_F32");
    int ndev = 0;
    MOT_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) MOT_FAIL(MOT_EINVAL, "device index out of range");
    MOT_CUDA_TRY(cudaSetDevice(device));
    int sms = 0;
    MOT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    const int threads = 256, blocks = sms * 8;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    DBuf out;
    mot_status rc = MOT_OK;
    auto launch = [&](int iters) -> float {
        float t = -1.f;
        if (cudaEventRecord(e0, st) != cudaSuccess) return t;
        count_launch();
        if (dtype == MOT_F64)
            k_fma_peak<double><<<blocks, threads, 0, st>>>((double *)out.p, iters, 0.999999, 1e-6);
        else
            k_fma_peak<float><<<blocks, threads, 0, st>>>((float *)out.p, iters, 0.999f, 1e-3f);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            return -1.f;
        return t;
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = MOT_ECUDA;
        set_error("stream or event creation failed");
    } else if ((rc = dalloc(out, sizeof(double) * (size_t)blocks * threads)) == MOT_OK) {
        // calibrate to about 100 ms per launch, then keep the best of three
        int iters = 64;
        float t = launch(iters);
        while (t >= 0.f && t < 20.f && iters < (1 << 24)) {
            iters *= 4;
            t = launch(iters);
        }
        if (t > 0.f) iters = (int)std::min<double>((double)(1 << 28), iters * (100.0 / t));
        float best = 1e30f;
        for (int rep = 0; rep < 3 && t >= 0.f; ++rep) {
            t = launch(iters);
            if (t > 0.f) best = std::min(best, t);
        }
        if (t < 0.f) {
            rc = MOT_ECUDA;
            set_error("FMA microkernel launch failed");
        } else {
            const double fmas = (double)blocks * threads * iters * 4.0 * kPeakChains;
            *flop_per_s = 2.0 * fmas / (best * 1e-3);
            if (ms) *ms = best;
        }
    }
    dfree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return rc;
}

mot_status mot_run_step_index(const mot_run *r, int64_t *n) {
    if (!r || !n) MOT_FAIL(MOT_EINVAL, "NULL argument");
    *n = r->n;
    return MOT_OK;
}

void mot_run_destroy(mot_run *r) {
    if (!r) return;
    cudaSetDevice(r->p->ctx->device);
    cudaStreamSynchronize(r->p->ctx->stream);
    dfree(r->pw);
    dfree(r->inc);
    dfree(r->J);
    dfree(r->J2);
    dfree(r->J3);
    dfree(r->b);
    dfree(r->r);
    dfree(r->ring);
    dfree(r->hacc);
    dfree(r->hpart);
    dfree(r->wsAh);
    dfree(r->wsBh);
    for (int i = 0; i < 10; ++i) dfree(r->kv[i]);
    dfree(r->r32);
    dfree(r->scal);
    dfree(r->part1);
    dfree(r->part2);
    dfree(r->part3);
    dfree(r->dots);
    for (int i = 0; i < 4; ++i)
        if (r->ev[i]) cudaEventDestroy(r->ev[i]);
    for (cudaEvent_t e : r->sev) cudaEventDestroy(e);
    if (r->jcopy) {
        cudaStreamSynchronize(r->jcopy);
        cudaStreamDestroy(r->jcopy);
    }
    for (int b = 0; b < 2; ++b) {
        dfree(r->jstage[b]);
        if (r->jready[b]) cudaEventDestroy(r->jready[b]);
        if (r->jdone[b]) cudaEventDestroy(r->jdone[b]);
    }
    for (LoopGraph *G : {&r->loop64, &r->loop32}) {
        if (G->exec) cudaGraphExecDestroy(G->exec);
        if (G->graph) cudaGraphDestroy(G->graph);
    }
    dfree(r->ctl);
    dfree(r->ctr);
    dfree(r->inctab);
    if (r->step_exec) cudaGraphExecDestroy(r->step_exec);
    if (r->step_graph) cudaGraphDestroy(r->step_graph);
    dfree(r->sdev);
    dfree(r->sstats);
    dfree(r->b2);
    dfree(r->r2);
    if (r->cap) cudaStreamDestroy(r->cap);
    if (r->cap2) cudaStreamDestroy(r->cap2);
    if (r->cap3) cudaStreamDestroy(r->cap3);
    if (r->hside) cudaStreamDestroy(r->hside);
    if (r->hfork) cudaEventDestroy(r->hfork);
    if (r->hjoin) cudaEventDestroy(r->hjoin);
    delete r;
}

}  // extern "C"

// ============================================================================
// Z0 product without allocation: scratch in a file-scope device array
// ============================================================================
// The array's device address is resolved once per device (host code cannot
// use the symbol itself as a device pointer).
static __device__ __align__(256) unsigned char g_static_scratch[MOT_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// device address of g_static_scratch per device ordinal, resolved on the first
// call on that device; atomic so that threads racing on a first call agree
std::atomic<void *> g_static_ptr[kMaxDevices];
}  // namespace

extern "C" mot_status mot_apply_Z0_static(mot_problem *p, const void *x_dev, void *y_dev, int nrhs, int dtype) {
    if (!p || !x_dev || !y_dev) MOT_FAIL(MOT_EINVAL, "NULL argument");
    if (nrhs < 1) MOT_FAIL(MOT_EINVAL, "nrhs < 1");
    if (dtype != MOT_F64 && dtype != MOT_F32 && dtype != MOT_F64DF)
        MOT_FAIL(MOT_EINVAL, "dtype must be MOT_F64, MOT_F32 or MOT_F64DF");
    if (x_dev == y_dev) MOT_FAIL(MOT_EINVAL, "x and y must not overlap");
    if ((reinterpret_cast<uintptr_t>(x_dev) | reinterpret_cast<uintptr_t>(y_dev)) & 15u)
        MOT_FAIL(MOT_EINVAL, "x and y must be 16-byte aligned");
    const int dev = p->ctx->device;
    if (dev < 0 || dev >= kMaxDevices) MOT_FAIL(MOT_EINVAL, "device index beyond the static-scratch table");
    size_t a, b;
    z0_ws_bytes(p, nrhs, dtype == MOT_F32 ? sizeof(float2) : sizeof(double2), &a, &b);
    a = (a + 255) / 256 * 256;
    if (a + b > (size_t)MOT_STATIC_SCRATCH_BYTES)
        MOT_FAIL(MOT_EINVAL, "mot_apply_Z0_static needs " + std::to_string(a + b) + " bytes of scratch; the static array holds " +
                                 std::to_string((size_t)MOT_STATIC_SCRATCH_BYTES));
    MOT_CUDA_TRY(cudaSetDevice(dev));
    void *ptr = g_static_ptr[dev].load(std::memory_order_acquire);
    if (!ptr) {
        MOT_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_static_scratch));
        g_static_ptr[dev].store(ptr, std::memory_order_release);
    }
    char *ws = (char *)ptr;
    const long pr = (long)p->N[2] * p->N[1];
    // this entry point records no kernel-timing events (the caller's stream may
    // be in a state where the library's own events must not be recorded)
    const bool was = p->capturing;
    p->capturing = true;
    // a schedule tuned earlier for this (nrhs, dtype) is used; none is tuned here
    SchedScope scope(p->sched_for(nrhs, dtype == MOT_F32));
    mot_status st;
    if (dtype == MOT_F64) {
        EpiZ0<double, double> e = {(const double *)x_dev, (double *)y_dev, eps_of<double>(p), pr, p->N[0],
                                   p->opt.delta};
        st = z0_product<double, double>(p, (const double *)x_dev, nrhs, ws, ws + a, e, p->ctx->stream);
    } else if (dtype == MOT_F64DF) {
        EpiZ0DF e = {(const double *)x_dev, (double *)y_dev, eps_of<double>(p), pr, p->N[0], p->opt.delta};
        st = z0_product<double, dfl>(p, (const double *)x_dev, nrhs, ws, ws + a, e, p->ctx->stream);
    } else {
        EpiZ0<float, float> e = {(const float *)x_dev, (float *)y_dev, eps_of<float>(p), pr, p->N[0],
                             (float)p->opt.delta};
        st = z0_product<float, float>(p, (const float *)x_dev, nrhs, ws, ws + a, e, p->ctx->stream);
    }
    p->capturing = was;
    return st;
}

// ---------------------------------------------------------------- serving
#include "server.cuh"
