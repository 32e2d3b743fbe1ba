// cufft_compare.cu -- comparison baseline for the Z0 product (Eq. 11-12) built
// on cuFFT: zero-pad each current component onto the M0 grid, cuFFT R2C (D2Z)
// of all 3 * nrhs components in one batched plan, one fused kernel for the 3x3
// real spectral multiply, cuFFT C2R (Z2D), one epilogue kernel for truncation
// and the contrast terms (y = eps T(0) x - (eps - 1) G x).
//
// Timed only, beside the library's own product; no part of the solver uses
// it.  Built into its own shared library (libmotcufft.so) so the solver
// library does not link cuFFT.  C ABI: status 0 on success, -1 bad argument,
// -2 allocation, -5 CUDA or cuFFT failure; mcf_last_error() describes it.
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <string>

namespace {

thread_local std::string g_err;

template <typename T> struct Cx;
template <> struct Cx<float> {
    using type = cufftComplex;
};
template <> struct Cx<double> {
    using type = cufftDoubleComplex;
};

struct Handle {
    int dev = 0, fp64 = 0, nrhs = 1;
    int N[3], M[3], H;
    cudaStream_t st = nullptr;
    cufftHandle fwd = 0, inv = 0;
    bool plans = false;
    void *pad = nullptr;   // [3 nrhs][Mz][My][Mx] real
    void *spec = nullptr;  // [3 nrhs][Mz][My][H] complex
    void *lam = nullptr;   // [6][Mz][My][H] real (xx yy zz xy xz yz), 1/(Mx My Mz) included
    void *eps = nullptr;   // [Nz][Ny][Nx] real
};

template <typename T>
__global__ void k_pad(const T *__restrict__ x, T *__restrict__ pad, int Nx, int Ny, int Nz, int Mx, int My, int Mz,
                      long total) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const int mx = (int)(i % Mx);
        const long r = i / Mx;
        const int my = (int)(r % My);
        const long r2 = r / My;
        const int mz = (int)(r2 % Mz);
        const long c = r2 / Mz;
        T v = T(0);
        if (mx < Nx && my < Ny && mz < Nz) v = x[((c * Nz + mz) * Ny + my) * Nx + mx];
        pad[i] = v;
    }
}

template <typename T>
__global__ void k_mul(typename Cx<T>::type *__restrict__ s, const T *__restrict__ lam, long nf, int nrhs) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nf * nrhs; i += (long)gridDim.x * blockDim.x) {
        const long f = i % nf, b = i / nf;
        const T l0 = lam[f], l1 = lam[nf + f], l2 = lam[2 * nf + f];
        const T l3 = lam[3 * nf + f], l4 = lam[4 * nf + f], l5 = lam[5 * nf + f];
        auto *p = s + 3 * b * nf + f;
        const auto X = p[0], Y = p[nf], Z = p[2 * nf];
        p[0].x = l0 * X.x + l3 * Y.x + l4 * Z.x;
        p[0].y = l0 * X.y + l3 * Y.y + l4 * Z.y;
        p[nf].x = l3 * X.x + l1 * Y.x + l5 * Z.x;
        p[nf].y = l3 * X.y + l1 * Y.y + l5 * Z.y;
        p[2 * nf].x = l4 * X.x + l5 * Y.x + l2 * Z.x;
        p[2 * nf].y = l4 * X.y + l5 * Y.y + l2 * Z.y;
    }
}

template <typename T>
__global__ void k_epi(const T *__restrict__ x, const T *__restrict__ g, const T *__restrict__ eps, T *__restrict__ y,
                      int Nx, int Ny, int Nz, int Mx, int My, int Mz, long total) {
    const long nv = (long)Nx * Ny * Nz;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long m = i % nv, c = i / nv;
        const int mx = (int)(m % Nx), my = (int)((m / Nx) % Ny), mz = (int)(m / ((long)Nx * Ny));
        const T gv = g[((c * Mz + mz) * My + my) * Mx + mx];
        const T e = eps[m];
        y[i] = e * T(0.5) * x[i] - (e - T(1)) * gv;
    }
}

unsigned grid_of(long n) {
    long g = (n + 255) / 256;
    if (g > 148L * 32) g = 148L * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

void destroy(Handle *h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->plans) {
        cufftDestroy(h->fwd);
        cufftDestroy(h->inv);
    }
    cudaFree(h->pad);
    cudaFree(h->spec);
    cudaFree(h->lam);
    cudaFree(h->eps);
    delete h;
}

}  // namespace

extern "C" {

const char *mcf_last_error(void) { return g_err.c_str(); }

// N = {Nx, Ny, Nz}, M = {Mx, My, Mz} (M_i >= N_i); lam: host [6][Mz][My][Mx/2+1]
// doubles (the real spectrum of the circulant lag-0 table, scaled by 1/(Mx My Mz));
// eps: host [Nz][Ny][Nx] doubles; stream borrowed (NULL = legacy default).
int mcf_create(int device, void *stream, const int32_t N[3], const int32_t M[3], int nrhs, int fp64, const double *lam,
               const double *eps, void **out) {
    if (!N || !M || !lam || !eps || !out || nrhs < 1) {
        g_err = "bad argument";
        return -1;
    }
    *out = nullptr;
    Handle *h = new Handle();
    h->dev = device;
    h->fp64 = fp64 ? 1 : 0;
    h->nrhs = nrhs;
    h->st = (cudaStream_t)stream;
    for (int i = 0; i < 3; ++i) {
        h->N[i] = N[i];
        h->M[i] = M[i];
        if (M[i] < N[i] || N[i] < 1) {
            g_err = "grid sizes";
            delete h;
            return -1;
        }
    }
    h->H = M[0] / 2 + 1;
    const size_t es = fp64 ? 8 : 4;
    const long nreal = (long)M[0] * M[1] * M[2], nspec = (long)M[2] * M[1] * h->H, nv = (long)N[0] * N[1] * N[2];
    auto fail = [&](int code, const char *msg) {
        g_err = msg;
        destroy(h);
        return code;
    };
    if (cudaSetDevice(device) != cudaSuccess) return fail(-5, "cudaSetDevice");
    if (cudaMalloc(&h->pad, es * 3 * nrhs * nreal) != cudaSuccess ||
        cudaMalloc(&h->spec, 2 * es * 3 * nrhs * nspec) != cudaSuccess ||
        cudaMalloc(&h->lam, es * 6 * nspec) != cudaSuccess || cudaMalloc(&h->eps, es * nv) != cudaSuccess) {
        cudaGetLastError();
        return fail(-2, "cudaMalloc");
    }
    if (fp64) {
        if (cudaMemcpy(h->lam, lam, 8 * 6 * nspec, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->eps, eps, 8 * nv, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(-5, "cudaMemcpy");
    } else {
        float *tl = new float[6 * nspec], *te = new float[nv];
        for (long i = 0; i < 6 * nspec; ++i) tl[i] = (float)lam[i];
        for (long i = 0; i < nv; ++i) te[i] = (float)eps[i];
        const bool ok = cudaMemcpy(h->lam, tl, 4 * 6 * nspec, cudaMemcpyHostToDevice) == cudaSuccess &&
                        cudaMemcpy(h->eps, te, 4 * nv, cudaMemcpyHostToDevice) == cudaSuccess;
        delete[] tl;
        delete[] te;
        if (!ok) return fail(-5, "cudaMemcpy");
    }
    int n[3] = {M[2], M[1], M[0]};
    int inembed[3] = {M[2], M[1], M[0]}, onembed[3] = {M[2], M[1], h->H};
    const int batch = 3 * nrhs;
    if (cufftPlanMany(&h->fwd, 3, n, inembed, 1, (int)nreal, onembed, 1, (int)nspec, fp64 ? CUFFT_D2Z : CUFFT_R2C,
                      batch) != CUFFT_SUCCESS)
        return fail(-5, "cufftPlanMany (forward)");
    if (cufftPlanMany(&h->inv, 3, n, onembed, 1, (int)nspec, inembed, 1, (int)nreal, fp64 ? CUFFT_Z2D : CUFFT_C2R,
                      batch) != CUFFT_SUCCESS) {
        cufftDestroy(h->fwd);
        return fail(-5, "cufftPlanMany (inverse)");
    }
    h->plans = true;
    cufftSetStream(h->fwd, h->st);
    cufftSetStream(h->inv, h->st);
    *out = h;
    return 0;
}

// y = Z0 x for nrhs current vectors [nrhs][3][Nz][Ny][Nx] of the handle's precision (device)
int mcf_apply(void *handle, const void *x, void *y) {
    Handle *h = (Handle *)handle;
    if (!h || !x || !y) {
        g_err = "bad argument";
        return -1;
    }
    cudaSetDevice(h->dev);
    const long nreal = (long)h->M[0] * h->M[1] * h->M[2], nspec = (long)h->M[2] * h->M[1] * h->H;
    const long nv = (long)h->N[0] * h->N[1] * h->N[2];
    const long tpad = 3L * h->nrhs * nreal, tvec = 3L * h->nrhs * nv;
    cufftResult r1, r2;
    if (h->fp64) {
        k_pad<double><<<grid_of(tpad), 256, 0, h->st>>>((const double *)x, (double *)h->pad, h->N[0], h->N[1], h->N[2],
                                                       h->M[0], h->M[1], h->M[2], tpad);
        r1 = cufftExecD2Z(h->fwd, (cufftDoubleReal *)h->pad, (cufftDoubleComplex *)h->spec);
        k_mul<double><<<grid_of(nspec * h->nrhs), 256, 0, h->st>>>((cufftDoubleComplex *)h->spec,
                                                                  (const double *)h->lam, nspec, h->nrhs);
        r2 = cufftExecZ2D(h->inv, (cufftDoubleComplex *)h->spec, (cufftDoubleReal *)h->pad);
        k_epi<double><<<grid_of(tvec), 256, 0, h->st>>>((const double *)x, (const double *)h->pad, (const double *)h->eps,
                                                       (double *)y, h->N[0], h->N[1], h->N[2], h->M[0], h->M[1],
                                                       h->M[2], tvec);
    } else {
        k_pad<float><<<grid_of(tpad), 256, 0, h->st>>>((const float *)x, (float *)h->pad, h->N[0], h->N[1], h->N[2],
                                                      h->M[0], h->M[1], h->M[2], tpad);
        r1 = cufftExecR2C(h->fwd, (cufftReal *)h->pad, (cufftComplex *)h->spec);
        k_mul<float><<<grid_of(nspec * h->nrhs), 256, 0, h->st>>>((cufftComplex *)h->spec, (const float *)h->lam, nspec,
                                                                 h->nrhs);
        r2 = cufftExecC2R(h->inv, (cufftComplex *)h->spec, (cufftReal *)h->pad);
        k_epi<float><<<grid_of(tvec), 256, 0, h->st>>>((const float *)x, (const float *)h->pad, (const float *)h->eps,
                                                      (float *)y, h->N[0], h->N[1], h->N[2], h->M[0], h->M[1], h->M[2],
                                                      tvec);
    }
    if (r1 != CUFFT_SUCCESS || r2 != CUFFT_SUCCESS || cudaGetLastError() != cudaSuccess) {
        g_err = "cuFFT or kernel launch failed";
        return -5;
    }
    return 0;
}

void mcf_destroy(void *handle) { destroy((Handle *)handle); }

}  // extern "C"
