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

__device__ __forceinline__ float block_sum_f(float v, float *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int t = threadIdx.y * blockDim.x + threadIdx.x;
    int lane = t & 31, warp = t >> 5, nw = (blockDim.x * blockDim.y + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float r = 0.0f;
    if (warp == 0) {
        r = lane < nw ? sh[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// FP64 residual rounded to FP32 as the right-hand side of the FP32 correction
// cycle (in the scaled form the correction equation's right-hand side is rho
// itself), with per-block partial sums of rho^2 for the stopping test.  The
// squares are summed in FP32: they only decide when to stop, and a relative
// error of 1e-7 in ||rho|| shifts the threshold by as much.
template <int OP>
__global__ void __launch_bounds__(kBX *kBY)
    k_residual64_to32(const double *__restrict__ psi, const double *__restrict__ g, int N, int P,
                      float *__restrict__ r32, int P32, double *__restrict__ partials, FinishArgs fin) {
    pdl_enter();
    __shared__ float sh[32];
    int i0 = 1 + blockIdx.x * kRX;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    float v = 0.0f;
    double rho;
    if (rho_halo<double, OP>(psi, g, N, P, i0, j, rho)) {
        float r = f64_to_f32(rho);
        r32[(size_t)j * P32 + i0 - 1 + (int)(threadIdx.x & 31)] = r;
        v = r * r;
    }
    v = block_sum_f(v, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = (double)v;
    if (fin.enabled) finish_if_last(partials, fin);
}

__global__ void __launch_bounds__(kBX *kBY)
    k_correct64(const float *__restrict__ e, int Pe, double *__restrict__ psi, int P64, float *__restrict__ psi32,
                int P32, int N) {
    pdl_enter();
    int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P64 + i;
    double p = psi[c] + f32_to_f64(e[(size_t)j * Pe + i]);
    psi[c] = p;
    if (psi32) psi32[(size_t)j * P32 + i] = f64_to_f32(p);
}

// L(omega) in FP32 from the FP32 shadows, stage combination in FP64 (see
// StageCoef); writes the FP64 stage vorticity and its FP32 shadow.
__global__ void __launch_bounds__(kBX *kBY)
    k_rhs_stage_mixed(const float *__restrict__ psi, int Ps, const float *__restrict__ in32,
                      const double *__restrict__ in64, const double *__restrict__ W0, double *__restrict__ acc,
                      double *__restrict__ out64, float *__restrict__ out32, int N, int P64, int P32, float inv2h,
                      float nu_invh2, int advect, StageCoef k) {
    pdl_enter();
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
    double Ld = f32_to_f64(L), wPd = in64[c64];
    double o;
    if (k.mode == 3) {
        o = fma(k.bdt, Ld, fma(k.a1, wPd, acc[c64]));
    } else {
        o = fma(k.bdt, Ld, fma(k.a1, wPd, k.a0 * W0[c64]));
        if (k.mode == 1) acc[c64] = k.acc_in * wPd;
        else if (k.mode == 2) acc[c64] = fma(k.acc_L, Ld, fma(k.acc_in, wPd, acc[c64]));
    }
    out64[c64] = o;
    out32[c] = f64_to_f32(o);
}

struct Walls {
    double *w64[3];
    float *w32[3];
};

// Thom's wall vorticity (Eq. (25)) in FP64 from psi64, written to the three
// FP64 stage buffers and their FP32 shadows.
__global__ void k_thom_mixed(const double *__restrict__ psi, Walls w, int N, int P64, int P32, double U, int profile) {
    pdl_enter();
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
        w.w32[b][(size_t)j * P32 + i] = f64_to_f32(val);
    }
}

__global__ void k_to32(const double *__restrict__ src, int P64, float *__restrict__ dst, int P32, int N) {
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > N || j > N) return;
    dst[(size_t)j * P32 + i] = f64_to_f32(src[(size_t)j * P64 + i]);
}

// ---------------------------------------------------------------------------
// Batched forms.  SSPRK(5,4) stage s reads stage buffer kIn[s] and writes
// kOut[s] (0 = W0, 1 = Wa, 2 = Wb; ACC is W[3]); the coefficients are those of
// the single-cavity step, with dt taken per cavity.
__device__ __forceinline__ int stage_in(int s) { return s == 0 ? 0 : (s & 1 ? 1 : 2); }     // 0,1,2,1,2
__device__ __forceinline__ int stage_out(int s) { return s == 4 ? 0 : (s & 1 ? 2 : 1); }   // 1,2,1,2,0

// RHS64: L(omega) in FP64 from psi64 and the FP64 stage vorticity (the
// shadows are then neither read nor written), as the FP64 step computes it.
template <bool RHS64>
__global__ void __launch_bounds__(kBX *kBY)
    k_stage_batch(const BatchCav *cav, const BatchRange *r, int stage, StageCoef k, int advect) {
    pdl_enter();
    int bx, by;
    const BatchCav &cv = cav[batch_locate(r, bx, by)];
    int N = cv.N, P = cv.P[0];
    int i = 1 + bx * kBX + threadIdx.x, j = 1 + by * kBY + threadIdx.y;
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P + i;
    const double *in64 = cv.W[stage_in(stage)], *W0 = cv.W[0];
    double *acc = cv.W[3], *out64 = cv.W[stage_out(stage)];
    double Ld, wPd = in64[c];
    if (RHS64) {
        const double *psi = cv.psi64;
        double inv2h = 0.5 * N, nu_invh2 = cv.nu_invh2;
        double wE = in64[c + 1], wW = in64[c - 1], wN = in64[c + P], wS = in64[c - P];
        Ld = nu_invh2 * fma(-4.0, wPd, (wE + wW) + (wN + wS));
        if (advect) {
            double u = (psi[c + P] - psi[c - P]) * inv2h;
            double v = -(psi[c + 1] - psi[c - 1]) * inv2h;
            double tx = u * ((wE - wW) * inv2h);
            double ty = v * ((wN - wS) * inv2h);
            Ld = (Ld - tx) - ty;
        }
    } else {
        const float *in32 = cv.Ws[stage_in(stage)], *psi = cv.psi32;
        float inv2h = 0.5f * (float)N;  // exact: the value (float)(0.5 N) of the single-cavity launcher
        float nu_invh2 = cv.nu_invh2f;
        float wP = in32[c], wE = in32[c + 1], wW = in32[c - 1], wN = in32[c + P], wS = in32[c - P];
        float L = nu_invh2 * fmaf(-4.0f, wP, (wE + wW) + (wN + wS));
        if (advect) {
            float u = (psi[c + P] - psi[c - P]) * inv2h;
            float v = -(psi[c + 1] - psi[c - 1]) * inv2h;
            float tx = u * ((wE - wW) * inv2h);
            float ty = v * ((wN - wS) * inv2h);
            L = (L - tx) - ty;
        }
        Ld = f32_to_f64(L);
    }
    double bdt = k.bdt * cv.dt, o;
    if (k.mode == 3) {
        o = fma(bdt, Ld, fma(k.a1, wPd, acc[c]));
    } else {
        o = fma(bdt, Ld, fma(k.a1, wPd, k.a0 * W0[c]));
        if (k.mode == 1) acc[c] = k.acc_in * wPd;
        else if (k.mode == 2) acc[c] = fma(k.acc_L * cv.dt, Ld, fma(k.acc_in, wPd, acc[c]));
    }
    out64[c] = o;
    if (!RHS64) cv.Ws[stage_out(stage)][c] = f64_to_f32(o);
}

// Poisson right-hand side (as k_assemble_rhs) of every cavity's new stage
// vorticity, per-block partial sums of g^2, and the start of each cavity's
// solve (all cavities iterate again).
template <int OP>
__global__ void __launch_bounds__(kBX *kBY)
    k_assemble_batch(BatchCav *cav, const BatchRange *r, int stage, double *__restrict__ gpart) {
    pdl_enter();
    __shared__ double sh[32];
    int bx, by;
    int ci = batch_locate(r, bx, by);
    BatchCav &cv = cav[ci];
    if (bx == 0 && by == 0 && threadIdx.x == 0 && threadIdx.y == 0) cv.active = 1;
    int N = cv.N, P = cv.P[0];
    const double *w = cv.W[stage_out(stage)];
    double h2 = cv.h2;
    int i = 1 + bx * kBX + threadIdx.x, j = 1 + by * kBY + threadIdx.y;
    double v = 0.0;
    if (i < N && j < N) {
        size_t c = (size_t)j * P + i;
        double val;
        if (OP == 1)
            val = h2 * fma(8.0, w[c], (w[c + 1] + w[c - 1]) + (w[c + P] + w[c - P])) * (1.0 / 40.0);
        else
            val = 0.25 * h2 * w[c];
        cv.g64[c] = val;
        v = val * val;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) gpart[blockIdx.x] = v;
}

// FP64 residual of every active cavity rounded to FP32 (as k_residual64_to32)
// with per-block partial sums of rho^2.  With fin.enabled, the last block of
// each cavity applies that cavity's stopping rule (same rule and summation
// order as the single-cavity finisher), and the last cavity to finish sets
// the loop condition: go on while any cavity iterates.
template <int OP>
__global__ void __launch_bounds__(kBX *kBY)
    k_residual_batch(BatchCav *cav, const BatchRange *r, const BatchRange *rg, double *__restrict__ rpart,
                     const double *__restrict__ gpart, BatchFinish fin) {
    pdl_enter();
    __shared__ double sh[32];
    __shared__ float shf[32];
    __shared__ unsigned int s_last;
    int bx, by;
    int ci = batch_locate(r, bx, by);
    BatchCav &cv = cav[ci];
    int N = cv.N, P = cv.P[0];
    int i0 = 1 + bx * kRX, j = 1 + by * kRY + threadIdx.y;
    float v = 0.0f;
    double rho;
    if (cv.active && rho_halo<double, OP>(cv.psi64, cv.g64, N, P, i0, j, rho)) {
        float rf = f64_to_f32(rho);
        cv.g32[0][(size_t)j * P + i0 - 1 + (int)(threadIdx.x & 31)] = rf;
        v = rf * rf;
    }
    v = block_sum_f(v, shf);
    int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    if (tid == 0) rpart[blockIdx.x] = (double)v;
    if (!fin.enabled) return;
    int b0 = r->start[ci], nb = r->start[ci + 1] - b0;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&cv.arrive, 1u) == (unsigned)nb - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (cv.active) {
        double sr = 0.0, sg = 0.0;
        int g0 = rg->start[ci], ng = rg->start[ci + 1] - g0;
        for (int k = tid; k < nb; k += nt) sr += __ldcg(rpart + b0 + k);
        for (int k = tid; k < ng; k += nt) sg += __ldcg(gpart + g0 + k);
        sr = block_sum(sr, sh);
        sg = block_sum(sg, sh);
        if (tid == 0) {
            int cyc = cv.cycles + 1;
            double rn = sqrt(sr), gn = sqrt(sg);
            bool finite = isfinite(rn) && isfinite(gn);
            bool more = false;
            if (!finite) {
                cv.status |= kStatusNonFinite;
            } else if (rn <= fin.tol * gn) {
            } else if (cyc >= fin.max_cycles) {
                cv.status |= kStatusNoConv;
            } else {
                more = true;
            }
            if (more) {
                cv.cycles = cyc;
            } else {
                cv.cycles = 0;
                cv.active = 0;
                cv.last_cycles = cyc;
                cv.last_rel = gn > 0.0 ? rn / gn : (rn > 0.0 ? INFINITY : 0.0);
                cv.log[cv.nsolves % kLogN] = cyc;
                cv.nsolves += 1;
            }
        }
    }
    if (tid != 0) return;
    cv.arrive = 0;
    __threadfence();
    if (atomicAdd(&fin.bs->cav_arrive, 1u) != (unsigned)r->count - 1) return;
    __threadfence();
    fin.bs->cav_arrive = 0;
    unsigned int any = 0;
    for (int c = 0; c < r->count; ++c) any |= (unsigned)((volatile BatchCav *)cav)[c].active;
    if (fin.h)
        cudaGraphSetConditional(fin.h, any ? 1u : 0u);
    else
        fin.bs->more = (int)any;
}

// FP32 shadow of every cavity's psi64 after its solve (read only by the next
// stage's FP32 L(omega)).
__global__ void __launch_bounds__(kBX *kBY) k_psi32_batch(const BatchCav *cav, const BatchRange *r) {
    pdl_enter();
    int bx, by;
    const BatchCav &cv = cav[batch_locate(r, bx, by)];
    int N = cv.N, P = cv.P[0];
    int i = 1 + bx * kBX + threadIdx.x, j = 1 + by * kBY + threadIdx.y;
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P + i;
    cv.psi32[c] = f64_to_f32(cv.psi64[c]);
}

// Thom's wall vorticity for every cavity (blockIdx.y = cavity), uniform lid U.
__global__ void k_thom_batch(const BatchCav *cav, double U) {
    pdl_enter();
    const BatchCav &cv = cav[blockIdx.y];
    int N = cv.N, P = cv.P[0];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int n = N - 1;
    double m2h2 = -2.0 * (double)N * (double)N;
    const double *psi = cv.psi64;
    int i, j;
    double val;
    if (t < n) {
        i = t + 1;
        j = 0;
        val = m2h2 * psi[(size_t)P + i];
    } else if (t < 2 * n) {
        i = t - n + 1;
        j = N;
        val = m2h2 * psi[(size_t)(N - 1) * P + i] - 2.0 * U * N;
    } else if (t < 3 * n) {
        j = t - 2 * n + 1;
        i = 0;
        val = m2h2 * psi[(size_t)j * P + 1];
    } else if (t < 4 * n) {
        j = t - 3 * n + 1;
        i = N;
        val = m2h2 * psi[(size_t)j * P + N - 1];
    } else if (t < 4 * n + 4) {
        int k = t - 4 * n;
        i = k & 1 ? N : 0;
        j = k & 2 ? N : 0;
        val = 0.0;
    } else {
        return;
    }
    for (int b = 0; b < 3; ++b) {
        cv.W[b][(size_t)j * P + i] = val;
        cv.Ws[b][(size_t)j * P + i] = f64_to_f32(val);
    }
}

}  // namespace

cudaError_t launch_stage_batch(cudaStream_t s, BatchCav *cav, const BatchRange *r, int nblocks, int stage,
                               int advect, int rhs64) {
    // SSPRK(5,4) stage coefficients, Eqs. (9)-(13): bdt and acc_L are scaled by each cavity's dt in the kernel
    static const StageCoef kc[5] = {
        {1.0, 0.0, 0.391752226571890, 0.0, 0.0, 0},
        {0.444370493651235, 0.555629506348765, 0.368410593050371, 0.0, 0.0, 0},
        {0.620101851488403, 0.379898148511597, 0.251891774271694, 0.517231671970585, 0.0, 1},
        {0.178079954393132, 0.821920045606868, 0.544974750228521, 0.096059710526147, 0.063692468666290, 2},
        {0.0, 0.386708617503269, 0.226007483236906, 0.0, 0.0, 3}};
    if (rhs64)
        (void)launch_pdl(k_stage_batch<true>, nblocks, dim3(kBX, kBY), 0, s, cav, r, stage, kc[stage], advect);
    else
        (void)launch_pdl(k_stage_batch<false>, nblocks, dim3(kBX, kBY), 0, s, cav, r, stage, kc[stage], advect);
    return cudaGetLastError();
}

cudaError_t launch_assemble_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, int nblocks, int stage,
                                  double *gpart) {
    if (op == 1)
        (void)launch_pdl(k_assemble_batch<1>, nblocks, dim3(kBX, kBY), 0, s, cav, r, stage, gpart);
    else
        (void)launch_pdl(k_assemble_batch<0>, nblocks, dim3(kBX, kBY), 0, s, cav, r, stage, gpart);
    return cudaGetLastError();
}

cudaError_t launch_residual_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, const BatchRange *rg,
                                  int nblocks, double *rpart, const double *gpart, BatchFinish fin) {
    if (op == 1)
        (void)launch_pdl(k_residual_batch<1>, nblocks, dim3(kBX, kRY), 0, s, cav, r, rg, rpart, gpart, fin);
    else
        (void)launch_pdl(k_residual_batch<0>, nblocks, dim3(kBX, kRY), 0, s, cav, r, rg, rpart, gpart, fin);
    return cudaGetLastError();
}

cudaError_t launch_psi32_batch(cudaStream_t s, BatchCav *cav, const BatchRange *r, int nblocks) {
    (void)launch_pdl(k_psi32_batch, nblocks, dim3(kBX, kBY), 0, s, cav, r);
    return cudaGetLastError();
}

cudaError_t launch_thom_batch(cudaStream_t s, BatchCav *cav, int count, double U) {
    // N <= 8192: 4 (N - 1) + 4 <= 32768 wall nodes
    (void)launch_pdl(k_thom_batch, dim3(32768 / 256, count), 256, 0, s, cav, U);
    return cudaGetLastError();
}

cudaError_t launch_residual64_to32(cudaStream_t s, int op, const double *psi64, const double *g64, int N, int P64,
                                   float *r32, int P32, double *partials, FinishArgs fin) {
    dim3 grid(residual_blocks_x(N), (N - 1 + kRY - 1) / kRY);
    if (op == 1)
        (void)launch_pdl(k_residual64_to32<1>, grid, dim3(kBX, kRY), 0, s, psi64, g64, N, P64, r32, P32, partials, fin);
    else
        (void)launch_pdl(k_residual64_to32<0>, grid, dim3(kBX, kRY), 0, s, psi64, g64, N, P64, r32, P32, partials, fin);
    return cudaGetLastError();
}

cudaError_t launch_correct64(cudaStream_t s, const float *e32, int Pe, double *psi64, int P64, float *psi32, int P32,
                             int N) {
    (void)launch_pdl(k_correct64, grid2(N - 1, N - 1), dim3(kBX, kBY), 0, s, e32, Pe, psi64, P64, psi32, P32, N);
    return cudaGetLastError();
}

cudaError_t launch_rhs_stage_mixed(cudaStream_t s, const float *psi32, int Ps, const float *in32, const double *in64,
                                   const double *W0, double *acc, double *out64, float *out32, int N, int P64, int P32,
                                   double Re, int advect, StageCoef c) {
    float inv2h = (float)(0.5 * N);
    float nu_invh2 = (float)((double)N * (double)N / Re);
    (void)launch_pdl(k_rhs_stage_mixed, grid2(N - 1, N - 1), dim3(kBX, kBY), 0, s, psi32, Ps, in32, in64, W0, acc,
                     out64, out32, N, P64, P32, inv2h, nu_invh2, advect, c);
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
    (void)launch_pdl(k_thom_mixed, (n + 255) / 256, 256, 0, s, psi64, w, N, P64, P32, U, profile);
    return cudaGetLastError();
}

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {  // SplitMix64 finaliser
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ bool same_bits_f(float a, float b) {
    return __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
}

__device__ __forceinline__ bool same_bits_d(double a, double b) {
    return __double_as_longlong(a) == __double_as_longlong(b) || (a != a && b != b);
}

// Value k of the conversion test: fixed edge cases first, then four kinds
// of generated FP64 patterns (raw 64-bit words; exponents around the FP32
// range with random mantissas; the same with the 29 rounded-off bits at or
// next to the halfway point; the FP32 subnormal range with ties at the
// subnormal rounding position) and FP32 patterns (raw, subnormal).
__device__ double conv_case(long long k, unsigned long long seed, float &f) {
    const double edge[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38, 3.4028235677973366e38,
                           3.4028235677973362e38, 3.4028235677973370e38, 6.805646932770577e38,
                           1.1754943508222875e-38, 1.1754942106924411e-38, 5.877471754111438e-39,
                           1.401298464324817e-45, 7.006492321624085e-46, 7.006492321624087e-46,
                           2.1019476964872256e-45, 4.9406564584124654e-324, 2.2250738585072014e-308,
                           1.7976931348623157e308, __longlong_as_double(0x7ff0000000000000ll),
                           __longlong_as_double(0xfff0000000000000ll), __longlong_as_double(0x7ff8000000000001ll),
                           0.1, 1.0 / 3.0, 1e-40, -1e-44};
    const int nedge = (int)(sizeof(edge) / sizeof(edge[0]));
    const unsigned long long u = mix64(seed ^ mix64((unsigned long long)k));
    f = __uint_as_float((unsigned)(u >> 7));
    if (k < nedge) {
        f = (float)edge[k];
        return edge[k];
    }
    const unsigned long long sign = u & 0x8000000000000000ull, mant = u & 0xfffffffffffffull;
    switch (k & 3) {
        case 0:
            if (k & 4) f = __uint_as_float((unsigned)(u >> 32) & 0x807fffffu);  // FP32 subnormals
            return __longlong_as_double((long long)u);
        case 1: {
            const unsigned long long e = 853 + ((u >> 52) & 0x7ffull) % 320;
            return __longlong_as_double((long long)(sign | (e << 52) | mant));
        }
        case 2: {
            const unsigned long long e = 853 + ((u >> 52) & 0x7ffull) % 320;
            const unsigned long long low[4] = {0x10000000ull, 0x0fffffffull, 0x10000001ull, 0ull};
            return __longlong_as_double((long long)(sign | (e << 52) | (mant & ~0x1fffffffull) | low[(u >> 40) & 3]));
        }
        default: {
            const unsigned long long e = 840 + ((u >> 52) & 0x7ffull) % 60;  // FP32 subnormal results
            const int sh = 926 - (int)e;
            unsigned long long m = mant;
            if (((u >> 41) & 1) && sh >= 1 && sh <= 52) m = (m & ~((1ull << sh) - 1)) | (1ull << (sh - 1));  // a tie
            m &= 0xfffffffffffffull;
            return __longlong_as_double((long long)(sign | (e << 52) | m));
        }
    }
}

__global__ void k_selftest_conversions(long long n, unsigned long long seed, unsigned long long *bad) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        float f;
        const double d = conv_case(k, seed, f);
        if (!same_bits_f(f64_to_f32(d), __double2float_rn(d))) atomicAdd(bad, 1ull);
        if (!same_bits_d(f32_to_f64(f), (double)f)) atomicAdd(bad + 1, 1ull);
    }
}

}  // namespace

cudaError_t launch_selftest_conversions(cudaStream_t s, long long n, unsigned long long seed,
                                        unsigned long long *bad) {
    k_selftest_conversions<<<1216, 256, 0, s>>>(n, seed, bad);
    return cudaGetLastError();
}

cudaError_t launch_to32(cudaStream_t s, const double *src, int P64, float *dst, int P32, int N) {
    (void)launch_pdl(k_to32, grid2(N + 1, N + 1), dim3(kBX, kBY), 0, s, src, P64, dst, P32, N);
    return cudaGetLastError();
}

}  // namespace lcx
