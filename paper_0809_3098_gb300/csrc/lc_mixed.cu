// Kernels of the mixed-precision step.
//
// The solution psi, the vorticity of every Runge-Kutta stage, the Poisson
// residual, the correction psi += e, Thom's wall vorticity (Eq. (25)) and the
// SSPRK(5,4) stage accumulation (Eqs. (9)-(13)) stay FP64; the multigrid
// V-cycle that computes e from the residual, and the stencil arithmetic of
// L(omega) (Eq. (8), velocities from Eq. (22)), run in FP32 on FP32 shadows of
// psi and omega.  This is iterative refinement of the Poisson solve: each
// outer iteration computes the FP64 residual r of L_h psi = f, one FP32
// V-cycle approximates L_h e = r, and psi += e in FP64, so the solve still
// stops at the FP64 relative residual tol (method: Cardoso & Bicudo,
// arXiv:0809.3098, Sec. 3).
#include "lc_internal.h"

namespace lcx {

namespace {

constexpr int kBX = 32, kBY = 8;

inline dim3 grid2(int nx, int ny) { return dim3((nx + kBX - 1) / kBX, (ny + kBY - 1) / kBY); }

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int t = threadIdx.y * blockDim.x + threadIdx.x;
    int lane = t & 31, warp = t >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// FP64 scaled residual rho = (Gauss-Seidel value) - psi at interior nodes,
// stored rounded to FP32 as the right-hand side of the FP32 correction cycle
// (in the scaled form the correction equation's right-hand side is rho
// itself), with per-block partial sums of rho^2 for the stopping test.
template <int OP>
__global__ void __launch_bounds__(kBX *kBY)
    k_residual64_to32(const double *__restrict__ psi, const double *__restrict__ g, int N, int P,
                      float *__restrict__ r32, int P32, double *__restrict__ partials, FinishArgs fin) {
    __shared__ double sh[32];
    int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    double v = 0.0;
    if (i < N && j < N) {
        size_t c = (size_t)j * P + i;
        double n4 = (psi[c + 1] + psi[c - 1]) + (psi[c + P] + psi[c - P]);
        double gs;
        if (OP == 1) {
            double d4 = (psi[c + P + 1] + psi[c + P - 1]) + (psi[c - P + 1] + psi[c - P - 1]);
            gs = fma(0.2, n4, fma(0.05, d4, g[c]));
        } else {
            gs = fma(0.25, n4, g[c]);
        }
        double rho = gs - psi[c];
        r32[(size_t)j * P32 + i] = (float)rho;
        v = rho * rho;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = v;
    if (fin.enabled) finish_if_last(partials, fin);
}

__global__ void __launch_bounds__(kBX *kBY)
    k_correct64(const float *__restrict__ e, int Pe, double *__restrict__ psi, int P64, float *__restrict__ psi32,
                int P32, int N) {
    int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P64 + i;
    double p = psi[c] + (double)e[(size_t)j * Pe + i];
    psi[c] = p;
    psi32[(size_t)j * P32 + i] = (float)p;
}

// L(omega) in FP32 from the FP32 shadows, stage combination in FP64 (see
// StageCoef); writes the FP64 stage vorticity and its FP32 shadow.
__global__ void __launch_bounds__(kBX *kBY)
    k_rhs_stage_mixed(const float *__restrict__ psi, int Ps, const float *__restrict__ in32,
                      const double *__restrict__ in64, const double *__restrict__ W0, double *__restrict__ acc,
                      double *__restrict__ out64, float *__restrict__ out32, int N, int P64, int P32, float inv2h,
                      float nu_invh2, int advect, StageCoef k) {
    int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P32 + i, cs = (size_t)j * Ps + i, c64 = (size_t)j * P64 + i;
    float wP = in32[c], wE = in32[c + 1], wW = in32[c - 1], wN = in32[c + P32], wS = in32[c - P32];
    float L = nu_invh2 * fmaf(-4.0f, wP, (wE + wW) + (wN + wS));
    if (advect) {
        float u = (psi[cs + Ps] - psi[cs - Ps]) * inv2h;
        float v = -(psi[cs + 1] - psi[cs - 1]) * inv2h;
        float tx = u * ((wE - wW) * inv2h);
        float ty = v * ((wN - wS) * inv2h);
        L = (L - tx) - ty;
    }
    double Ld = (double)L, wPd = in64[c64];
    double o;
    if (k.mode == 3) {
        o = fma(k.bdt, Ld, fma(k.a1, wPd, acc[c64]));
    } else {
        o = fma(k.bdt, Ld, fma(k.a1, wPd, k.a0 * W0[c64]));
        if (k.mode == 1) acc[c64] = k.acc_in * wPd;
        else if (k.mode == 2) acc[c64] = fma(k.acc_L, Ld, fma(k.acc_in, wPd, acc[c64]));
    }
    out64[c64] = o;
    out32[c] = (float)o;
}

struct Walls {
    double *w64[3];
    float *w32[3];
};

// Thom's wall vorticity (Eq. (25)) in FP64 from psi64, written to the three
// FP64 stage buffers and their FP32 shadows.
__global__ void k_thom_mixed(const double *__restrict__ psi, Walls w, int N, int P64, int P32, double U, int profile) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int n = N - 1;
    double m2h2 = -2.0 * (double)N * (double)N;
    int i, j;
    double val;
    if (t < n) {
        i = t + 1;
        j = 0;
        val = m2h2 * psi[(size_t)P64 + i];
    } else if (t < 2 * n) {
        i = t - n + 1;
        j = N;
        double x = i * (1.0 / N);
        double ui = profile == 1 ? U * 16.0 * x * x * (1.0 - x) * (1.0 - x) : U;
        val = m2h2 * psi[(size_t)(N - 1) * P64 + i] - 2.0 * ui * N;
    } else if (t < 3 * n) {
        j = t - 2 * n + 1;
        i = 0;
        val = m2h2 * psi[(size_t)j * P64 + 1];
    } else if (t < 4 * n) {
        j = t - 3 * n + 1;
        i = N;
        val = m2h2 * psi[(size_t)j * P64 + N - 1];
    } else if (t < 4 * n + 4) {
        int k = t - 4 * n;
        i = k & 1 ? N : 0;
        j = k & 2 ? N : 0;
        val = 0.0;
    } else {
        return;
    }
    for (int b = 0; b < 3; ++b) {
        w.w64[b][(size_t)j * P64 + i] = val;
        w.w32[b][(size_t)j * P32 + i] = (float)val;
    }
}

__global__ void k_to32(const double *__restrict__ src, int P64, float *__restrict__ dst, int P32, int N) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > N || j > N) return;
    dst[(size_t)j * P32 + i] = (float)src[(size_t)j * P64 + i];
}

}  // namespace

cudaError_t launch_residual64_to32(cudaStream_t s, int op, const double *psi64, const double *g64, int N, int P64,
                                   float *r32, int P32, double *partials, FinishArgs fin) {
    if (op == 1)
        k_residual64_to32<1><<<grid2(N - 1, N - 1), dim3(kBX, kBY), 0, s>>>(psi64, g64, N, P64, r32, P32, partials,
                                                                              fin);
    else
        k_residual64_to32<0><<<grid2(N - 1, N - 1), dim3(kBX, kBY), 0, s>>>(psi64, g64, N, P64, r32, P32, partials,
                                                                              fin);
    return cudaGetLastError();
}

cudaError_t launch_correct64(cudaStream_t s, const float *e32, int Pe, double *psi64, int P64, float *psi32, int P32,
                             int N) {
    k_correct64<<<grid2(N - 1, N - 1), dim3(kBX, kBY), 0, s>>>(e32, Pe, psi64, P64, psi32, P32, N);
    return cudaGetLastError();
}

cudaError_t launch_rhs_stage_mixed(cudaStream_t s, const float *psi32, int Ps, const float *in32, const double *in64,
                                   const double *W0, double *acc, double *out64, float *out32, int N, int P64, int P32,
                                   double Re, int advect, StageCoef c) {
    float inv2h = (float)(0.5 * N);
    float nu_invh2 = (float)((double)N * (double)N / Re);
    k_rhs_stage_mixed<<<grid2(N - 1, N - 1), dim3(kBX, kBY), 0, s>>>(psi32, Ps, in32, in64, W0, acc, out64, out32, N,
                                                                      P64, P32, inv2h, nu_invh2, advect, c);
    return cudaGetLastError();
}

cudaError_t launch_thom_mixed(cudaStream_t s, const double *psi64, double *const w64[3], float *const w32[3], int N,
                              int P64, int P32, double U, int profile) {
    Walls w;
    for (int b = 0; b < 3; ++b) {
        w.w64[b] = w64[b];
        w.w32[b] = w32[b];
    }
    int n = 4 * (N - 1) + 4;
    k_thom_mixed<<<(n + 255) / 256, 256, 0, s>>>(psi64, w, N, P64, P32, U, profile);
    return cudaGetLastError();
}

cudaError_t launch_to32(cudaStream_t s, const double *src, int P64, float *dst, int P32, int N) {
    k_to32<<<grid2(N + 1, N + 1), dim3(kBX, kBY), 0, s>>>(src, P64, dst, P32, N);
    return cudaGetLastError();
}

}  // namespace lcx
