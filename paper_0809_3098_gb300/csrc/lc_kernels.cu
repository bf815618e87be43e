// CUDA kernels of the cavity step (sm_103a).
//
// Method: Cardoso & Bicudo, arXiv:0809.3098.  Poisson: compact operator of
// Sec. 3, Eq. (14), smoothed by the SOR update of Eq. (15) in colour order
// inside a multigrid V-cycle; Thom's wall vorticity, Sec. 3.1, Eq. (25);
// L(omega), Sec. 3, Eq. (8) with velocities from Eq. (22); SSPRK(5,4) stage
// combination, Eqs. (9)-(13); RES monitors, Sec. 3.2, Eqs. (26)-(27).
//
// All stencils are bandwidth- or FP64-ALU-bound; none is a dense contraction,
// so no tensor-core path is used.  Sums of mirror-image neighbours are always
// paired ((E + W) + (N + S)) so that the discrete scheme stays exactly
// equivariant under x -> 1 - x with (psi, omega, U) -> (-psi, -omega, -U).
#include "lc_internal.h"

#include <cooperative_groups.h>

#include <cmath>

namespace lcx {

thread_local int tl_pdl = 0;

namespace {

constexpr int kBX = 32, kBY = 8;

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (warp == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
    }
    return r;
}

// Gauss-Seidel value at node c of the scaled operator (see lc_internal.h).
template <typename T, int OP>
__device__ __forceinline__ T gs_value(const T *__restrict__ psi, const T *__restrict__ g, size_t c, int P) {
    T n4 = (psi[c + 1] + psi[c - 1]) + (psi[c + P] + psi[c - P]);
    if (OP == 1) {
        T d4 = (psi[c + P + 1] + psi[c - P + 1]) + (psi[c + P - 1] + psi[c - P - 1]);
        return fma(T(0.2), n4, fma(T(0.05), d4, g[c]));
    }
    return fma(T(0.25), n4, g[c]);
}

// ---------------------------------------------------------------------------
// One colour phase of the SOR smoother, Eq. (15).  Compact: colour
// (i mod 2) + 2 (j mod 2); 5-point: colour (i + j) mod 2.  Nodes of one colour
// never neighbour each other, so the phase is a Jacobi update of that colour.
// Each thread updates two nodes of the colour in one column, rows j and j+2,
// which share the loads of row j+1; RELAX = false is the beta = 1 update.
// Compact: the lanes of a warp hold same-colour nodes two columns apart in one
// row, so the diagonal sum d4 = V(i+1) + V(i-1), with the column sums
// V(k) = psi(k, j+1) + psi(k, j-1), takes V(i-1) from the lane to the left
// (the same additions in the same order as gs_value, one fewer per node).
// Lane 0 of each warp only supplies that column sum to lane 1 and updates no
// node: computing its own left sum would be a warp-wide FP64 instruction for
// one lane, as dear on GB300 (~64 clocks) as one for all 32.
//
// colour_item does the work of thread (a, b) of a phase (a: the colour
// node's column index, b: its row pair); the lanes of a warp must hold
// consecutive a of one b, for the compact operator a = 31 w + lane - 1 (lane
// 0 the halo, see colour_a).  L2 = true reads psi through L2 (for the fused
// kernel, whose blocks read values other blocks wrote in the same launch).
template <bool L2, typename T>
__device__ __forceinline__ T ldp(const T *p) {
    return L2 ? __ldcg(p) : *p;
}

// Colour column index of lane `lane` of warp-sized item w of a row: 31 nodes
// per warp for the compact operator (lane 0 a halo), 32 for the 5-point one.
template <int OP>
__device__ __forceinline__ int colour_a(int w, int lane) {
    return OP == 1 ? 31 * w + lane - 1 : 32 * w + lane;
}
template <int OP>
__host__ __device__ constexpr int colour_per_warp() {
    return OP == 1 ? 31 : 32;
}

template <typename T, int OP, bool RELAX, bool L2>
__device__ __forceinline__ void colour_item(T *psi, const T *__restrict__ g, int N, int P, int colour, T beta, int a,
                                            int b) {
    int i, j;
    if (OP == 1) {
        i = ((colour & 1) ? 1 : 2) + 2 * a;
        j = ((colour >> 1) ? 1 : 2) + 4 * b;  // rows j and j + 2
    } else {
        // thread rows (1,3), (2,4), (5,7), (6,8), ...: j and j + 2 share a parity
        j = 1 + 4 * (b >> 1) + (b & 1);
        i = (((colour + j) & 1) ? 1 : 2) + 2 * a;
    }
    if (OP == 1) {
        // every lane of the warp reaches the shuffles; lanes past the grid
        // load nothing and store nothing
        bool rowok = j < N, ok = rowok && i < N && (threadIdx.x & 31) != 0;
        bool second = ok && j + 2 < N;
        size_t c = (size_t)j * P + i, c2 = c + 2 * (size_t)P;
        bool colr = rowok && i + 1 <= N;  // column i + 1 exists (it may be the wall)
        T m_e = colr ? ldp<L2>(psi + c + P + 1) : T(0);
        T m_c = ok ? ldp<L2>(psi + c + P) : T(0);
        T Vr = colr ? m_e + ldp<L2>(psi + c - P + 1) : T(0);
        T V2r = (colr && j + 2 < N) ? ldp<L2>(psi + c2 + P + 1) + m_e : T(0);
        T Vl = __shfl_up_sync(0xffffffffu, Vr, 1), V2l = __shfl_up_sync(0xffffffffu, V2r, 1);
        if (!ok) return;
        T n4 = (ldp<L2>(psi + c + 1) + ldp<L2>(psi + c - 1)) + (m_c + ldp<L2>(psi + c - P));
        T v1 = fma(T(0.2), n4, fma(T(0.05), Vr + Vl, g[c])), v2 = T(0);
        if (second) {
            T n42 = (ldp<L2>(psi + c2 + 1) + ldp<L2>(psi + c2 - 1)) + (ldp<L2>(psi + c2 + P) + m_c);
            v2 = fma(T(0.2), n42, fma(T(0.05), V2r + V2l, g[c2]));
        }
        if (RELAX) {
            T o1 = ldp<L2>(psi + c);
            v1 = fma(beta, v1 - o1, o1);
            if (second) {
                T o2 = ldp<L2>(psi + c2);
                v2 = fma(beta, v2 - o2, o2);
            }
        }
        psi[c] = v1;
        if (second) psi[c2] = v2;
        return;
    }
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P + i;
    bool second = j + 2 < N;
    size_t c2 = c + 2 * (size_t)P;
    T m_c = ldp<L2>(psi + c + P);  // shared row j + 1
    T v1 = fma(T(0.25), (ldp<L2>(psi + c + 1) + ldp<L2>(psi + c - 1)) + (m_c + ldp<L2>(psi + c - P)), g[c]),
      v2 = T(0);
    if (second)
        v2 = fma(T(0.25), (ldp<L2>(psi + c2 + 1) + ldp<L2>(psi + c2 - 1)) + (ldp<L2>(psi + c2 + P) + m_c), g[c2]);
    if (RELAX) {
        T o1 = ldp<L2>(psi + c);
        v1 = fma(beta, v1 - o1, o1);
        if (second) {
            T o2 = ldp<L2>(psi + c2);
            v2 = fma(beta, v2 - o2, o2);
        }
    }
    psi[c] = v1;
    if (second) psi[c2] = v2;
}

template <typename T, int OP, bool RELAX>
__global__ void __launch_bounds__(kBX *kBY)
    k_smooth_colour(T *__restrict__ psi, const T *__restrict__ g, int N, int P, int colour, T beta) {
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;  // blockDim.x = 32: one warp per block row
    colour_item<T, OP, RELAX, false>(psi, g, N, P, colour, beta, colour_a<OP>(t >> 5, t & 31),
                                     blockIdx.y * blockDim.y + threadIdx.y);
}

// Grid-wide barrier between the colour phases of a cooperative launch (all
// blocks co-resident).  The arrival count only grows within a launch: barrier
// k (k = 1, 2, ...) releases once it reaches k * expected, so an arrival is
// one fence and one atomic add whose result nobody waits for, and a waiter
// polls one word with acquire loads; nothing is reset between phases.  The
// last block to leave the kernel (exit count, ds->bar_gen) sets both words
// back to zero for the next launch.  Every wait is bounded: after kBarCycles
// SM clock cycles (about 0.2 s) a block gives up, sets kStatusTimeout
// (reported as LC_ERR_TIMEOUT) and goes on, so the kernel always ends.
// `expected` is the number of arrivals per barrier (gridDim.x; one more only
// in the test that makes the wait run out).
constexpr long long kBarCycles = 400000000LL;
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void grid_barrier(DevState *ds, unsigned target) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // the block's writes (ordered before by the block barrier) before the arrival
        atomicAdd(&ds->bar_count, 1u);
        long long t0 = clock64();
        while ((int)(ld_acquire_gpu(&ds->bar_count) - target) < 0) {
            if (clock64() - t0 > kBarCycles) {
                atomicOr(&ds->status, kStatusTimeout);
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Called once by every block as its last action: the last block out resets
// the barrier words for the next launch.
__device__ __forceinline__ void grid_barrier_exit(DevState *ds) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ds->bar_gen, 1u) == gridDim.x - 1) {
            ds->bar_count = 0;
            ds->bar_gen = 0;
            __threadfence();
        }
    }
}

// nsweeps colour sweeps of the smoother in one cooperative launch: the
// threads of phase (a, b) of k_smooth_colour become warp-sized items (a warp:
// 32 consecutive a of one b); each block takes an equal contiguous share of
// the items, so the SMs get equal FP64 work, and a grid barrier separates the
// phases.  Same per-node expression and colour order as the one-launch-per-
// phase form, so the same bits, without a launch per phase.
template <typename T, int OP, bool RELAX>
__global__ void __launch_bounds__(256)
    k_smooth_fused(T *psi, const T *__restrict__ g, int N, int P, int nsweeps, T beta, DevState *ds, int extra) {
    const int na = N / 2;                              // colour nodes per row: at most N / 2
    const int nb = OP == 1 ? (N / 2 + 1) / 2 : N / 2;  // row pairs
    const int nchunk = (na + colour_per_warp<OP>() - 1) / colour_per_warp<OP>(), items = nchunk * nb;
    const int lo = (int)((long long)items * blockIdx.x / gridDim.x);
    const int hi = (int)((long long)items * (blockIdx.x + 1) / gridDim.x);
    const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int ncol = OP == 1 ? 4 : 2;
    const unsigned expected = gridDim.x + extra;
    unsigned k = 0;  // barriers passed in this launch
    for (int s = 0; s < nsweeps; ++s)
        for (int col = 0; col < ncol; ++col) {
            if (s > 0 || col > 0) grid_barrier(ds, ++k * expected);
            for (int w = lo + wib; w < hi; w += nwb) {
                int b = w / nchunk, a = colour_a<OP>(w - b * nchunk, lane);
                colour_item<T, OP, RELAX, true>(psi, g, N, P, col, beta, a, b);
            }
        }
    grid_barrier_exit(ds);
}

// Residual of the fine level, full-weighted onto the coarse level; also zeroes
// the coarse correction (its initial guess).  A 16x16 block of coarse nodes
// needs the fine residual on a 33x33 patch, computed once into shared memory.
constexpr int kRT = 16;
template <typename T, int OP>
__global__ void __launch_bounds__(kRT *kRT)
    k_residual_restrict(const T *__restrict__ psi, const T *__restrict__ g, int Nf, int Pf, T *__restrict__ gc,
                        T *__restrict__ psic, int Pc) {
    pdl_enter();
    constexpr int kW = 2 * kRT + 1;  // the fine patch is kW x kW nodes
    __shared__ T rho[kW][kW + 1];
    int Nc = Nf / 2;
    int I0 = 1 + blockIdx.x * kRT, J0 = 1 + blockIdx.y * kRT;
    int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;
    int t = threadIdx.y * kRT + threadIdx.x;
    if constexpr (OP == 1 && sizeof(T) == 8) {
        // rho_node's H-form with each column sum V and H = 4 psi + V formed
        // once per node of the patch (plus one column on each side) and
        // shared by the three residuals that use it: six FP64 operations per
        // node instead of nine, the same values
        __shared__ T sV[kW][kW + 2], sH[kW][kW + 2];
        for (int k = t; k < kW * (kW + 2); k += kRT * kRT) {
            int x = k % (kW + 2), y = k / (kW + 2);
            int i = fi0 - 1 + x, j = fj0 + y;
            T V = T(0), H = T(0);
            if (i <= Nf && j < Nf) {
                size_t c = (size_t)j * Pf + i;
                V = psi[c + Pf] + psi[c - Pf];
                H = fma(T(4), psi[c], V);
            }
            sV[y][x] = V;
            sH[y][x] = H;
        }
        __syncthreads();
        for (int k = t; k < kW * kW; k += kRT * kRT) {
            int x = k % kW, y = k / kW;
            int i = fi0 + x, j = fj0 + y;
            T r = T(0);
            if (i < Nf && j < Nf) {
                size_t c = (size_t)j * Pf + i;
                r = fma(T(0.05), fma(T(4), sV[y][x + 1], sH[y][x + 2] + sH[y][x]), g[c] - psi[c]);
            }
            rho[y][x] = r;
        }
    } else {
        for (int k = t; k < kW * kW; k += kRT * kRT) {
            int x = k % kW, y = k / kW;
            int i = fi0 + x, j = fj0 + y;
            T r = T(0);
            if (i >= 1 && i < Nf && j >= 1 && j < Nf) {
                size_t c = (size_t)j * Pf + i;
                r = rho_node<T, OP>(psi, g, c, Pf);
            }
            rho[y][x] = r;
        }
    }
    __syncthreads();
    int I = I0 + threadIdx.x, J = J0 + threadIdx.y;
    if (I >= Nc || J >= Nc) return;
    int x = 2 * threadIdx.x + 1, y = 2 * threadIdx.y + 1;
    T e4 = (rho[y][x + 1] + rho[y][x - 1]) + (rho[y + 1][x] + rho[y - 1][x]);
    T d4 = (rho[y + 1][x + 1] + rho[y + 1][x - 1]) + (rho[y - 1][x + 1] + rho[y - 1][x - 1]);
    size_t cc = (size_t)J * Pc + I;
    gc[cc] = fma(T(0.5), e4, fma(T(0.25), d4, rho[y][x]));
    psic[cc] = T(0);
}

// Bilinear prolongation of the coarse correction onto fine node (i, j), added to psi.
template <typename T>
__device__ __forceinline__ void prolong_node(T *__restrict__ psi, int Pf, const T *__restrict__ ec, int Pc, int i,
                                             int j) {
    int I = i >> 1, J = j >> 1;
    size_t cc = (size_t)J * Pc + I;
    T e;
    if (!(i & 1) && !(j & 1))
        e = ec[cc];
    else if (i & 1 && !(j & 1))
        e = mul_rn(T(0.5), ec[cc] + ec[cc + 1]);
    else if (!(i & 1) && (j & 1))
        e = mul_rn(T(0.5), ec[cc] + ec[cc + Pc]);
    else
        e = mul_rn(T(0.25), (ec[cc] + ec[cc + 1]) + (ec[cc + Pc] + ec[cc + Pc + 1]));
    size_t c = (size_t)j * Pf + i;
    psi[c] = add_rn(psi[c], e);
}

// Bilinear prolongation of the coarse correction, added to the fine field.
// A block covers 64 columns x 8 rows; the lanes of a warp take every other
// column of one row in each of two passes, so a warp's nodes share one
// (i, j) parity and take one branch: the four parity classes need 0-3 FP64
// operations, and on GB300 a divergent branch costs its full warp-wide FP64
// issue (~64 clocks) per instruction whatever its lane count.
template <typename T>
__global__ void __launch_bounds__(kBX *kBY)
    k_prolong_correct(T *__restrict__ psi, int Nf, int Pf, const T *__restrict__ ec, int Pc) {
    pdl_enter();
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (j >= Nf) return;
    for (int p = 0; p < 2; ++p) {
        const int i = 1 + p + blockIdx.x * (2 * blockDim.x) + 2 * threadIdx.x;
        if (i < Nf) prolong_node<T>(psi, Pf, ec, Pc, i, j);
    }
}

// Coarsest grid (2, 3, 5 or 7 intervals: at most 36 unknowns, one thread each
// in a block of 64): nsweeps colour sweeps in one block.
template <typename T, int OP>
__global__ void k_coarsest(T *__restrict__ psi, const T *__restrict__ g, int N, int P, int nsweeps, T beta) {
    pdl_enter();
    int n = N - 1;
    int t = threadIdx.x;
    int i = 1 + t % n, j = 1 + t / n;
    bool active = t < n * n;
    int my_colour = OP == 1 ? (i & 1) + 2 * (j & 1) : (i + j) & 1;
    int ncol = OP == 1 ? 4 : 2;
    for (int s = 0; s < nsweeps; ++s)
        for (int colour = 0; colour < ncol; ++colour) {
            if (active && my_colour == colour) {
                size_t c = (size_t)j * P + i;
                T v = gs_value<T, OP>(psi, g, c, P);
                if (beta != T(1)) v = fma(beta, v - psi[c], psi[c]);
                psi[c] = v;
            }
            __syncthreads();
        }
}

// Per-block partial sums of rho^2 over interior nodes (FP64 accumulation); a
// block of 32 x 8 threads covers 30 x (8 kNormRows) interior nodes (rho_halo:
// the outer lanes of each warp are halo).  Each thread accumulates kNormRows
// rows, kRY apart, before the block sum: the sum's FP64 additions are warp
// instructions of ~64 clocks each on GB300 however few lanes they serve, so
// one reduction per kNormRows rows instead of one per row.
template <typename T, int OP>
__global__ void __launch_bounds__(kBX *kBY)
    k_residual_norm(const T *__restrict__ psi, const T *__restrict__ g, int N, int P, double *__restrict__ partials,
                    FinishArgs fin) {
    pdl_enter();
    __shared__ double sh[32];
    int i0 = 1 + blockIdx.x * kRX;
    int j0 = 1 + blockIdx.y * (kRY * kNormRows) + threadIdx.y;
    double v = 0.0;
#pragma unroll
    for (int k = 0; k < kNormRows; ++k) {  // warp-uniform: rho_halo's shuffles see every lane
        T rho;
        if (rho_halo<T, OP>(psi, g, N, P, i0, j0 + k * kRY, rho)) {
            double r = (double)rho;
            v = fma(r, r, v);
        }
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = v;
    if (fin.enabled) finish_if_last(partials, fin);
}

// Scaled Poisson right-hand side at the fine level from omega:
//   compact: g = kappa h^2 B = h^2 (sum(edge omega) + 8 omega_P) / 40  (B of Eq. (17))
//   5-point: g = h^2 omega_P / 4
// and per-block partial sums of g^2.
template <int OP>
__global__ void __launch_bounds__(kBX *kBY)
    k_assemble_rhs(const double *__restrict__ w, double *__restrict__ g, int N, int P, double h2,
                   double *__restrict__ gpart) {
    pdl_enter();
    __shared__ double sh[32];
    int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    double v = 0.0;
    if (i < N && j < N) {
        size_t c = (size_t)j * P + i;
        double val;
        if (OP == 1)
            val = h2 * fma(8.0, w[c], (w[c + 1] + w[c - 1]) + (w[c + P] + w[c - P])) * (1.0 / 40.0);
        else
            val = 0.25 * h2 * w[c];
        g[c] = val;
        v = val * val;
    }
    v = block_sum(v, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) gpart[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

// Thom's wall vorticity, Eq. (25): -2 psi_adjacent / h^2 on every wall, minus
// 2 U(x) / h on the lid; corners 0.  Written to all three vorticity buffers so
// that every stage buffer carries the latest (lagged) walls.
__global__ void k_thom(const double *__restrict__ psi, double *W0, double *Wa, double *Wb, int N, int P, double U,
                       int profile) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int n = N - 1;
    double m2h2 = -2.0 * (double)N * (double)N;
    size_t idx;
    double val;
    if (t < n) {
        int i = t + 1;
        idx = i;
        val = m2h2 * psi[(size_t)P + i];
    } else if (t < 2 * n) {
        int i = t - n + 1;
        double x = i * (1.0 / N);
        double ui = profile == 1 ? U * 16.0 * x * x * (1.0 - x) * (1.0 - x) : U;
        idx = (size_t)N * P + i;
        val = m2h2 * psi[(size_t)(N - 1) * P + i] - 2.0 * ui * N;
    } else if (t < 3 * n) {
        int j = t - 2 * n + 1;
        idx = (size_t)j * P;
        val = m2h2 * psi[(size_t)j * P + 1];
    } else if (t < 4 * n) {
        int j = t - 3 * n + 1;
        idx = (size_t)j * P + N;
        val = m2h2 * psi[(size_t)j * P + N - 1];
    } else if (t < 4 * n + 4) {
        int k = t - 4 * n;
        idx = (k & 1 ? (size_t)N : 0) + (k & 2 ? (size_t)N * P : 0);
        val = 0.0;
    } else {
        return;
    }
    W0[idx] = val;
    Wa[idx] = val;
    Wb[idx] = val;
}

// Fused L(omega) (Eq. (8), velocities from Eq. (22)) and SSPRK(5,4) stage
// combination (Eqs. (9)-(13)) in low-storage form (StageCoef).
__global__ void __launch_bounds__(kBX *kBY)
    k_rhs_stage(const double *__restrict__ psi, const double *__restrict__ in, const double *__restrict__ W0,
                double *__restrict__ acc, double *__restrict__ out, int N, int P, double inv2h, double nu_invh2,
                int advect, StageCoef k) {
    pdl_enter();
    int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= N || j >= N) return;
    size_t c = (size_t)j * P + i;
    double wP = in[c], wE = in[c + 1], wW = in[c - 1], wN = in[c + P], wS = in[c - P];
    double L = nu_invh2 * fma(-4.0, wP, (wE + wW) + (wN + wS));
    if (advect) {
        double u = (psi[c + P] - psi[c - P]) * inv2h;
        double v = -(psi[c + 1] - psi[c - 1]) * inv2h;
        double tx = u * ((wE - wW) * inv2h);
        double ty = v * ((wN - wS) * inv2h);
        L = (L - tx) - ty;
    }
    double o;
    if (k.mode == 3) {
        o = fma(k.bdt, L, fma(k.a1, wP, acc[c]));
    } else {
        o = fma(k.bdt, L, fma(k.a1, wP, k.a0 * W0[c]));
        if (k.mode == 1) acc[c] = k.acc_in * wP;
        else if (k.mode == 2) acc[c] = fma(k.acc_L, L, fma(k.acc_in, wP, acc[c]));
    }
    out[c] = o;
}

// Steady-state monitors between two states over all nodes: per-block max
// |d omega|, sum |d psi|, sum |d omega|; the last block to finish reduces the
// partials in block order.
__global__ void __launch_bounds__(kBX *kBY)
    k_monitor(const double *__restrict__ p0, const double *__restrict__ p1, const double *__restrict__ w0,
              const double *__restrict__ w1, int N, int P, double *__restrict__ part, unsigned int *counter,
              DevState *ds, double dt) {
    pdl_enter();
    __shared__ double sh[32];
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    double dw = 0.0, dp = 0.0;
    if (i <= N && j <= N) {
        size_t c = (size_t)j * P + i;
        dw = fabs(w1[c] - w0[c]);
        dp = fabs(p1[c] - p0[c]);
    }
    double mx = block_max(dw, sh);
    double sw = block_sum(dw, sh);
    double sp = block_sum(dp, sh);
    int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        part[3 * b] = mx;
        part[3 * b + 1] = sp;
        part[3 * b + 2] = sw;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    int t = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    double a = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = t; k < nb; k += nt) {
        a = fmax(a, ((volatile double *)part)[3 * k]);
        s1 += ((volatile double *)part)[3 * k + 1];
        s2 += ((volatile double *)part)[3 * k + 2];
    }
    a = block_max(a, sh);
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (t == 0) {
        ds->mon[0] = a / dt;
        ds->mon[1] = s1 / (N + 1);
        ds->mon[2] = s2 / (N + 1);
        if (!isfinite(a) || !isfinite(s1) || !isfinite(s2)) ds->status |= kStatusNonFinite;
        *counter = 0;
    }
}

__global__ void k_zero_walls(double *psi, int N, int P) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > N) return;
    psi[t] = 0.0;
    psi[(size_t)N * P + t] = 0.0;
    psi[(size_t)t * P] = 0.0;
    psi[(size_t)t * P + N] = 0.0;
}

inline dim3 grid2(int nx, int ny, int bx, int by) { return dim3((nx + bx - 1) / bx, (ny + by - 1) / by); }

}  // namespace

// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_smooth_colour(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int colour, T beta) {
    // Two-warp blocks: a phase is about one wave of work, and small blocks
    // spread it evenly over the SMs.
    constexpr int kSmY = 2;
    dim3 blk(kBX, kSmY);
    bool relax = beta != T(1);
    if (op == 1) {
        int n = N / 2;  // at most this many nodes of one parity per direction
        dim3 grid((n + colour_per_warp<1>() - 1) / colour_per_warp<1>(), ((n + 1) / 2 + kSmY - 1) / kSmY);
        if (relax)
            (void)launch_pdl(k_smooth_colour<T, 1, true>, grid, blk, 0, s, psi, g, N, P, colour, beta);
        else
            (void)launch_pdl(k_smooth_colour<T, 1, false>, grid, blk, 0, s, psi, g, N, P, colour, beta);
    } else {
        dim3 grid = grid2(N / 2, N / 2, kBX, kSmY);  // two rows per thread
        if (relax)
            (void)launch_pdl(k_smooth_colour<T, 0, true>, grid, blk, 0, s, psi, g, N, P, colour, beta);
        else
            (void)launch_pdl(k_smooth_colour<T, 0, false>, grid, blk, 0, s, psi, g, N, P, colour, beta);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_restrict(cudaStream_t s, int op, const T *psi, const T *g, int Nf, int Pf, T *gc, T *psic,
                                     int Pc) {
    int nc = Nf / 2 - 1;
    dim3 grid((nc + kRT - 1) / kRT, (nc + kRT - 1) / kRT), blk(kRT, kRT);
    if (op == 1)
        (void)launch_pdl(k_residual_restrict<T, 1>, grid, blk, 0, s, psi, g, Nf, Pf, gc, psic, Pc);
    else
        (void)launch_pdl(k_residual_restrict<T, 0>, grid, blk, 0, s, psi, g, Nf, Pf, gc, psic, Pc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_correct(cudaStream_t s, T *psi, int Nf, int Pf, const T *ec, int Pc) {
    (void)launch_pdl(k_prolong_correct<T>, grid2(Nf - 1, Nf - 1, 2 * kBX, kBY), dim3(kBX, kBY), 0, s, psi, Nf, Pf,
                     ec, Pc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int nsweeps, T beta) {
    if (op == 1)
        (void)launch_pdl(k_coarsest<T, 1>, 1, 64, 0, s, psi, g, N, P, nsweeps, beta);
    else
        (void)launch_pdl(k_coarsest<T, 0>, 1, 64, 0, s, psi, g, N, P, nsweeps, beta);
    return cudaGetLastError();
}

int residual_norm_blocks(int N) { return residual_blocks_x(N) * ((N - 1 + kRY - 1) / kRY); }
int residual_norm64_blocks(int N) {
    return residual_blocks_x(N) * ((N - 1 + kRY * kNormRows - 1) / (kRY * kNormRows));
}
int assemble_blocks(int N) { return ((N - 1 + kBX - 1) / kBX) * ((N - 1 + kBY - 1) / kBY); }
int monitor_blocks(int N) { return ((N + 1 + kBX - 1) / kBX) * ((N + 1 + kBY - 1) / kBY); }

template <typename T>
cudaError_t launch_residual_norm(cudaStream_t s, int op, const T *psi, const T *g, int N, int P, double *partials,
                                 FinishArgs fin) {
    dim3 grid(residual_blocks_x(N), (N - 1 + kRY * kNormRows - 1) / (kRY * kNormRows)), blk(kBX, kRY);
    if (op == 1)
        (void)launch_pdl(k_residual_norm<T, 1>, grid, blk, 0, s, psi, g, N, P, partials, fin);
    else
        (void)launch_pdl(k_residual_norm<T, 0>, grid, blk, 0, s, psi, g, N, P, partials, fin);
    return cudaGetLastError();
}

cudaError_t launch_assemble_rhs(cudaStream_t s, int op, const double *omega, double *g, int N, int P,
                                double *gpart) {
    double h = 1.0 / N;
    dim3 grid = grid2(N - 1, N - 1, kBX, kBY), blk(kBX, kBY);
    if (op == 1)
        (void)launch_pdl(k_assemble_rhs<1>, grid, blk, 0, s, omega, g, N, P, h * h, gpart);
    else
        (void)launch_pdl(k_assemble_rhs<0>, grid, blk, 0, s, omega, g, N, P, h * h, gpart);
    return cudaGetLastError();
}

cudaError_t launch_thom(cudaStream_t s, const double *psi, double *W0, double *Wa, double *Wb, int N, int P, double U,
                        int profile) {
    int n = 4 * (N - 1) + 4;
    (void)launch_pdl(k_thom, (n + 255) / 256, 256, 0, s, psi, W0, Wa, Wb, N, P, U, profile);
    return cudaGetLastError();
}

cudaError_t launch_rhs_stage(cudaStream_t s, const double *psi, const double *in, const double *W0, double *acc,
                             double *out, int N, int P, double Re, int advect, StageCoef c) {
    double inv2h = 0.5 * N;
    double nu_invh2 = (double)N * (double)N / Re;
    (void)launch_pdl(k_rhs_stage, grid2(N - 1, N - 1, kBX, kBY), dim3(kBX, kBY), 0, s, psi, in, W0, acc, out, N, P,
                     inv2h, nu_invh2, advect, c);
    return cudaGetLastError();
}

cudaError_t launch_monitor(cudaStream_t s, const double *psi0, const double *psi1, const double *w0,
                           const double *w1, int N, int P, double *part, DevState *ds, double dt) {
    // the block counter lives just past the partials
    unsigned int *counter = reinterpret_cast<unsigned int *>(part + 3 * monitor_blocks(N));
    (void)launch_pdl(k_monitor, grid2(N + 1, N + 1, kBX, kBY), dim3(kBX, kBY), 0, s, psi0, psi1, w0, w1, N, P, part,
                     counter, ds, dt);
    return cudaGetLastError();
}

cudaError_t launch_zero_walls(cudaStream_t s, double *psi, int N, int P) {
    (void)launch_pdl(k_zero_walls, (N + 1 + 255) / 256, 256, 0, s, psi, N, P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lexicographic SOR, Eq. (15) in the order its n / n+1 superscripts fix: at
// node (i, j) the neighbours (i-1, j-1), (i-1, j), (i-1, j+1) and (i, j-1)
// already hold this sweep's values, the others the previous sweep's (i is the
// outer loop, j the inner one).
//
// Wavefronts.  Number the interior nodes by t = W i + j (W = 2 compact, 1
// 5-point).  Every new neighbour of (i, j) lies on an earlier front (t - 1 ..
// t - 3) and every old one on a later front, and no two nodes of one front
// are neighbours.  Updating the fronts in increasing t, each front all at
// once, is therefore exactly the lexicographic sweep.  Sweep k + 1 may run D
// fronts behind sweep k (D = 4 compact, 2 5-point: one more than the
// stencil's reach in t), so nsw sweeps run as one pipelined pass of
// (number of fronts) + D (nsw - 1) steps, one barrier per step.  The method
// is sequential beyond a front, so one block does the pass when the grid fits
// its shared memory (psi updated in place there); larger grids use the
// cluster form below.  The node update is the smoother's expression.
template <int OP>
__device__ __forceinline__ double sor_value(const double *p, const double *__restrict__ g, size_t c, int P) {
    double n4 = (p[c + 1] + p[c - 1]) + (p[c + P] + p[c - P]);
    if (OP == 1) {
        double d4 = (p[c + P + 1] + p[c - P + 1]) + (p[c + P - 1] + p[c - P - 1]);
        return fma(0.2, n4, fma(0.05, d4, g[c]));
    }
    return fma(0.25, n4, g[c]);
}

template <int OP>
__global__ void __launch_bounds__(1024)
    k_sor_lex(double *psi, const double *__restrict__ g, int N, int P, int nsw, double beta) {
    pdl_enter();
    extern __shared__ double sor_sp[];
    double *p = sor_sp;
    const size_t nodes = (size_t)(N + 1) * P;
    for (size_t q = threadIdx.x; q < nodes; q += blockDim.x) p[q] = psi[q];
    __syncthreads();
    constexpr int W = OP == 1 ? 2 : 1, D = OP == 1 ? 4 : 2;
    const int t0 = W + 1, t1 = (W + 1) * (N - 1);
    const int maxc = (N - 2) / W + 1;  // most nodes on one front
    const int steps = (t1 - t0 + 1) + D * (nsw - 1);
    for (int s = 0; s < steps; ++s) {
        for (int q = threadIdx.x; q < nsw * maxc; q += blockDim.x) {
            int k = q / maxc, r = q - k * maxc;
            int t = t0 + s - D * k;
            if (t < t0 || t > t1) continue;
            int lo = t - (N - 1) > 0 ? (t - (N - 1) + W - 1) / W : 1;
            if (lo < 1) lo = 1;
            int i = lo + r, j = t - W * i;
            if (i > N - 1 || j < 1) continue;
            size_t c = (size_t)j * P + i;
            double v = sor_value<OP>(p, g, c, P);
            if (beta != 1.0) v = fma(beta, v - p[c], p[c]);
            p[c] = v;
        }
        __syncthreads();
    }
    for (size_t q = threadIdx.x; q < nodes; q += blockDim.x) psi[q] = p[q];
}

// Cluster form of the same pass for grids that do not fit one block's shared
// memory: the kSorCluster blocks of one thread-block cluster (co-scheduled on
// kSorCluster SMs, so the FP64 work of a step is spread over that many SMs)
// share each step's nodes, with a cluster barrier (release / acquire at
// cluster scope) between steps.  psi stays in global memory and is read and
// written through L2 (ld/st.global.cg), so no block sees a stale L1 copy of a
// node another block wrote.
constexpr int kSorCluster = 8;
// Dynamic shared memory requested (and not used) by each block of the
// cluster: more than half an SM's, so that no two blocks share an SM's FP64
// pipe.
constexpr int kSorClusterSmem = 120 * 1024;

template <int OP>
__device__ __forceinline__ double sor_value_l2(const double *p, const double *__restrict__ g, size_t c, int P) {
    double n4 = (__ldcg(p + c + 1) + __ldcg(p + c - 1)) + (__ldcg(p + c + P) + __ldcg(p + c - P));
    if (OP == 1) {
        double d4 = (__ldcg(p + c + P + 1) + __ldcg(p + c - P + 1)) + (__ldcg(p + c + P - 1) + __ldcg(p + c - P - 1));
        return fma(0.2, n4, fma(0.05, d4, g[c]));
    }
    return fma(0.25, n4, g[c]);
}

template <int OP>
__global__ void __launch_bounds__(1024)
    k_sor_lex_cluster(double *psi, const double *__restrict__ g, int N, int P, int nsw, double beta) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int nthreads = kSorCluster * (int)blockDim.x;
    const int tid = (int)cl.block_rank() * (int)blockDim.x + (int)threadIdx.x;
    constexpr int W = OP == 1 ? 2 : 1, D = OP == 1 ? 4 : 2;
    const int t0 = W + 1, t1 = (W + 1) * (N - 1);
    const int maxc = (N - 2) / W + 1;
    const int steps = (t1 - t0 + 1) + D * (nsw - 1);
    for (int s = 0; s < steps; ++s) {
        for (int q = tid; q < nsw * maxc; q += nthreads) {
            int k = q / maxc, r = q - k * maxc;
            int t = t0 + s - D * k;
            if (t < t0 || t > t1) continue;
            int lo = t - (N - 1) > 0 ? (t - (N - 1) + W - 1) / W : 1;
            if (lo < 1) lo = 1;
            int i = lo + r, j = t - W * i;
            if (i > N - 1 || j < 1) continue;
            size_t c = (size_t)j * P + i;
            double v = sor_value_l2<OP>(psi, g, c, P);
            if (beta != 1.0) {
                double o = __ldcg(psi + c);
                v = fma(beta, v - o, o);
            }
            __stcg(psi + c, v);
        }
        cl.sync();
    }
}

template <int OP>
cudaError_t launch_sor_cluster(cudaStream_t s, double *psi, const double *g, int N, int P, int nsw, double beta) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kSorCluster);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = kSorClusterSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSorCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sor_lex_cluster<OP>, psi, g, N, P, nsw, beta);
}

size_t sor_smem_bytes(int N, int P) { return (size_t)(N + 1) * P * sizeof(double); }

cudaError_t launch_sor_lex(cudaStream_t s, int op, double *psi, const double *g, int N, int P, int nsw, double beta) {
    size_t sm = sor_smem_bytes(N, P);
    if (sm > (size_t)kMaxSmem)
        return op == 1 ? launch_sor_cluster<1>(s, psi, g, N, P, nsw, beta)
                       : launch_sor_cluster<0>(s, psi, g, N, P, nsw, beta);
    if (op == 1)
        (void)launch_pdl(k_sor_lex<1>, 1, 1024, sm, s, psi, g, N, P, nsw, beta);
    else
        (void)launch_pdl(k_sor_lex<0>, 1, 1024, sm, s, psi, g, N, P, nsw, beta);
    return cudaGetLastError();
}

cudaError_t init_sor_kernel_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_sor_lex<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sor_lex<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sor_lex_cluster<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSorClusterSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sor_lex_cluster<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSorClusterSmem);
    return e;
}

template <typename T, int OP, bool RELAX>
static cudaError_t fused_t(cudaStream_t s, T *psi, const T *g, int N, int P, int nsweeps, T beta, DevState *ds,
                           int blocks, int extra) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_smooth_fused<T, OP, RELAX>, psi, g, N, P, nsweeps, beta, ds, extra);
}

template <typename T>
cudaError_t launch_smooth_fused(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int nsweeps, T beta,
                                DevState *ds, int blocks, int extra) {
    bool relax = beta != T(1);
    if (op == 1)
        return relax ? fused_t<T, 1, true>(s, psi, g, N, P, nsweeps, beta, ds, blocks, extra)
                     : fused_t<T, 1, false>(s, psi, g, N, P, nsweeps, beta, ds, blocks, extra);
    return relax ? fused_t<T, 0, true>(s, psi, g, N, P, nsweeps, beta, ds, blocks, extra)
                 : fused_t<T, 0, false>(s, psi, g, N, P, nsweeps, beta, ds, blocks, extra);
}
template cudaError_t launch_smooth_fused<double>(cudaStream_t, int, double *, const double *, int, int, int, double,
                                                 DevState *, int, int);

int smooth_fused_level_blocks(int op, int N, int nmax) {
    const int na = N / 2, nb = op == 1 ? (N / 2 + 1) / 2 : N / 2;
    const int per = op == 1 ? colour_per_warp<1>() : colour_per_warp<0>();
    const int items = ((na + per - 1) / per) * nb;  // warp-sized items of k_smooth_fused
    const int want = (items + 7) / 8;         // one item per warp of a 256-thread block
    return want < 1 ? 1 : (want < nmax ? want : nmax);
}

int smooth_fused_blocks(int op, bool relax) {
    int dev = 0, coop = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const void *k = op == 1 ? (relax ? (const void *)k_smooth_fused<double, 1, true> : (const void *)k_smooth_fused<double, 1, false>)
                            : (relax ? (const void *)k_smooth_fused<double, 0, true> : (const void *)k_smooth_fused<double, 0, false>);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, 256, 0) != cudaSuccess) return 0;
    // two blocks per SM: enough warps to keep the FP64 pipe busy, few barrier arrivals
    return (per < 2 ? per : 2) * sms;
}

#define LCX_INSTANTIATE(T)                                                                                           \
    template cudaError_t launch_smooth_colour<T>(cudaStream_t, int, T *, const T *, int, int, int, T);               \
    template cudaError_t launch_residual_restrict<T>(cudaStream_t, int, const T *, const T *, int, int, T *, T *,    \
                                                     int);                                                           \
    template cudaError_t launch_prolong_correct<T>(cudaStream_t, T *, int, int, const T *, int);                     \
    template cudaError_t launch_coarsest<T>(cudaStream_t, int, T *, const T *, int, int, int, T);                    \
    template cudaError_t launch_residual_norm<T>(cudaStream_t, int, const T *, const T *, int, int, double *,         \
                                                 FinishArgs);
LCX_INSTANTIATE(double)
LCX_INSTANTIATE(float)

}  // namespace lcx
