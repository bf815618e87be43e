// Register-tile ("warp tile") forms of the FP32 multigrid tile kernels: tile
// shape 4, 44 x 20 owned nodes per warp.
//
// The shared-memory tile kernels of lc_mg.cu separate every colour phase of
// the SOR smoother (Eq. (15), Cardoso & Bicudo, arXiv:0809.3098, Sec. 3) by a
// block barrier and read every neighbour from shared memory.  Here one warp
// owns a whole frame of 64 columns x 32 rows in registers: lane l holds
// columns 2l and 2l + 1 of every row, so the vertical neighbours of a node are
// in the same thread and the horizontal ones one lane away (warp shuffles).
// A colour phase needs no barrier and no shared memory at all; warps never
// wait on one another.  As in the shared-memory kernels, the frame recomputes
// a halo around the owned nodes (invalid values enter from the frame edge and
// spread one neighbour per colour phase, so after nu sweeps the residual is
// exact at distance >= (4 nu + 1, 2 nu + 1) from the edge for the compact
// operator, (2 nu + 1, 2 nu + 1) for the 5-point one); the frame fits that
// halo for nu <= 2.  Every node is computed with the expression and operand
// order of the shared-memory kernels (sums of mirror-image neighbours paired,
// the diagonal sum as V(i+1) + V(i-1) with the column sums V(k) = psi(k, j+1)
// + psi(k, j-1)), so the results are bit-identical to theirs.
#include "lc_internal.h"

namespace lcx {

namespace {

constexpr int kWF = 64;              // frame columns (lane l: 2l, 2l + 1)
constexpr int kWH = 32;              // frame rows, all in registers
constexpr int kWOX = 44, kWOY = 20;  // owned nodes per warp tile
constexpr int kWarps = 4;            // warp tiles per block
constexpr unsigned kFull = 0xffffffffu;

__host__ __device__ inline int whalo_x(int op, int nu) { return op == 1 ? 4 * nu + 1 : 2 * nu + 1; }
__host__ __device__ inline int whalo_y(int nu) { return 2 * nu + 1; }

// The frame holds the halo on both sides of the owned block plus the extra
// column / row of the restriction's residual.
__host__ __device__ inline bool warp_fits(int op, int nu) {
    return 2 * whalo_x(op, nu) + kWOX + 1 <= kWF && 2 * whalo_y(nu) + kWOY + 1 <= kWH;
}

struct WTile {
    int N, P, gx0, gy0, HX, HY, lane;
    bool u0, u1;      // this lane's columns may be updated (domain interior, not the frame edge)
    bool in0, in1;    // this lane's columns are domain-interior
    unsigned rows;    // bit y: frame row y is domain-interior and not a frame edge
};

__device__ __forceinline__ WTile wtile(int N, int P, int tx, int ty, int op, int nu) {
    WTile t;
    t.N = N;
    t.P = P;
    t.HX = whalo_x(op, nu);
    t.HY = whalo_y(nu);
    t.gx0 = 1 + tx * kWOX - t.HX;  // even: the owned block starts at an odd column, the halo is odd
    t.gy0 = 1 + ty * kWOY - t.HY;
    t.lane = threadIdx.x & 31;
    int i0 = t.gx0 + 2 * t.lane;
    t.in0 = i0 >= 1 && i0 <= N - 1;
    t.in1 = i0 + 1 >= 1 && i0 + 1 <= N - 1;
    t.u0 = t.in0 && t.lane != 0;
    t.u1 = t.in1 && t.lane != 31;
    t.rows = 0;
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y)
        if (t.gy0 + y >= 1 && t.gy0 + y <= N - 1) t.rows |= 1u << y;
    return t;
}

// Loads the frame of array a (zero outside [0, N]^2); pairs of columns as one
// 8-byte load where both are inside.
__device__ __forceinline__ void wload(const WTile &t, const float *__restrict__ a, float (&c0)[kWH],
                                      float (&c1)[kWH]) {
    int i0 = t.gx0 + 2 * t.lane;
    bool ok0 = i0 >= 0 && i0 <= t.N, ok1 = i0 + 1 >= 0 && i0 + 1 <= t.N;
#pragma unroll
    for (int y = 0; y < kWH; ++y) {
        int gj = t.gy0 + y;
        float v0 = 0.f, v1 = 0.f;
        if (gj >= 0 && gj <= t.N) {
            const float *row = a + (size_t)gj * t.P;
            if (ok0 && ok1) {
                float2 v = __ldg(reinterpret_cast<const float2 *>(row + i0));
                v0 = v.x;
                v1 = v.y;
            } else {
                if (ok0) v0 = __ldg(row + i0);
                if (ok1) v1 = __ldg(row + i0 + 1);
            }
        }
        c0[y] = v0;
        c1[y] = v1;
    }
}

// Compact operator, one colour phase: columns of parity PA (local parity =
// global parity, the frame starts at an even column), rows of local parity RP.
template <int PA, int RP, bool RELAX>
__device__ __forceinline__ void wphase_c(const WTile &t, float (&e0)[kWH], float (&e1)[kWH], const float (&g0)[kWH],
                                         const float (&g1)[kWH], float beta) {
#pragma unroll
    for (int y = (RP == 0 ? 2 : 1); y < kWH - 1; y += 2) {
        if (PA == 0) {
            float V1 = e1[y + 1] + e1[y - 1];              // V(2l + 1)
            float Vl = __shfl_up_sync(kFull, V1, 1);       // V(2l - 1)
            float W = __shfl_up_sync(kFull, e1[y], 1);
            float n4 = (e1[y] + W) + (e0[y + 1] + e0[y - 1]);
            float v = fmaf(0.2f, n4, fmaf(0.05f, V1 + Vl, g0[y]));
            if (RELAX) v = fmaf(beta, v - e0[y], e0[y]);
            if (t.u0 && (t.rows >> y & 1u)) e0[y] = v;
        } else {
            float V0 = e0[y + 1] + e0[y - 1];              // V(2l)
            float Vr = __shfl_down_sync(kFull, V0, 1);     // V(2l + 2)
            float E = __shfl_down_sync(kFull, e0[y], 1);
            float n4 = (E + e0[y]) + (e1[y + 1] + e1[y - 1]);
            float v = fmaf(0.2f, n4, fmaf(0.05f, Vr + V0, g1[y]));
            if (RELAX) v = fmaf(beta, v - e1[y], e1[y]);
            if (t.u1 && (t.rows >> y & 1u)) e1[y] = v;
        }
    }
}

// 5-point operator, one colour phase: node (i, j) has colour (i + j) mod 2;
// in frame row y the colour's column parity is (Q + y) mod 2.
template <int Q, bool RELAX>
__device__ __forceinline__ void wphase_5(const WTile &t, float (&e0)[kWH], float (&e1)[kWH], const float (&g0)[kWH],
                                         const float (&g1)[kWH], float beta) {
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y) {
        if (((Q + y) & 1) == 0) {
            float W = __shfl_up_sync(kFull, e1[y], 1);
            float v = fmaf(0.25f, (e1[y] + W) + (e0[y + 1] + e0[y - 1]), g0[y]);
            if (RELAX) v = fmaf(beta, v - e0[y], e0[y]);
            if (t.u0 && (t.rows >> y & 1u)) e0[y] = v;
        } else {
            float E = __shfl_down_sync(kFull, e0[y], 1);
            float v = fmaf(0.25f, (E + e0[y]) + (e1[y + 1] + e1[y - 1]), g1[y]);
            if (RELAX) v = fmaf(beta, v - e1[y], e1[y]);
            if (t.u1 && (t.rows >> y & 1u)) e1[y] = v;
        }
    }
}

// nu sweeps in the colour order of the other smoother kernels.
template <int OP, bool RELAX>
__device__ __forceinline__ void wsweeps(const WTile &t, float (&e0)[kWH], float (&e1)[kWH], const float (&g0)[kWH],
                                        const float (&g1)[kWH], int nu, float beta) {
    int gyp = t.gy0 & 1;
    for (int s = 0; s < nu; ++s) {
        if (OP == 1) {
            // colour c = (i mod 2) + 2 (j mod 2); local row parity = (c >> 1) ^ (gy0 mod 2)
            if (gyp == 0) {
                wphase_c<0, 0, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_c<1, 0, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_c<0, 1, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_c<1, 1, RELAX>(t, e0, e1, g0, g1, beta);
            } else {
                wphase_c<0, 1, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_c<1, 1, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_c<0, 0, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_c<1, 0, RELAX>(t, e0, e1, g0, g1, beta);
            }
        } else {
            // colour c: column parity in frame row y is (c + gy0 + y) mod 2
            if (gyp == 0) {
                wphase_5<0, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_5<1, RELAX>(t, e0, e1, g0, g1, beta);
            } else {
                wphase_5<1, RELAX>(t, e0, e1, g0, g1, beta);
                wphase_5<0, RELAX>(t, e0, e1, g0, g1, beta);
            }
        }
    }
}

template <int OP>
__device__ __forceinline__ void wsmooth(const WTile &t, float (&e0)[kWH], float (&e1)[kWH], const float (&g0)[kWH],
                                        const float (&g1)[kWH], int nu, float beta) {
    if (beta != 1.0f)
        wsweeps<OP, true>(t, e0, e1, g0, g1, nu, beta);
    else
        wsweeps<OP, false>(t, e0, e1, g0, g1, nu, beta);
}

// Writes the owned nodes of the frame.
__device__ __forceinline__ void wstore(const WTile &t, const float (&e0)[kWH], const float (&e1)[kWH],
                                       float *__restrict__ out) {
    int x0 = 2 * t.lane;
    bool o0 = t.in0 && x0 >= t.HX && x0 < t.HX + kWOX, o1 = t.in1 && x0 + 1 >= t.HX && x0 + 1 < t.HX + kWOX;
    int i0 = t.gx0 + x0;
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y) {
        if (!(t.rows >> y & 1u) || (unsigned)(y - t.HY) >= (unsigned)kWOY) continue;
        float *row = out + (size_t)(t.gy0 + y) * t.P;
        if (o0 && o1)
            *reinterpret_cast<float2 *>(row + i0) = make_float2(e0[y], e1[y]);
        else {
            if (o0) row[i0] = e0[y];
            if (o1) row[i0 + 1] = e1[y];
        }
    }
}

// ---------------------------------------------------------------------------
// Pre-smoothing from a zero correction, residual, full weighting onto the
// coarse grid (g_c = 4 R(rho)): k_down's work for one warp tile.
template <int OP, int GYP>
__device__ __forceinline__ void wrestrict(const WTile &t, const float (&r0)[kWH], const float (&r1)[kWH],
                                          float *__restrict__ gc, int Pc) {
    int Nc = t.N / 2;
    int x = 2 * t.lane;  // coarse nodes sit on even (global and local) columns
    bool colown = x >= t.HX && x < t.HX + kWOX;
    int I = (t.gx0 + x) >> 1;
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y) {
        if (((GYP + y) & 1) != 0) continue;  // coarse rows: even global row
        float Lc = __shfl_up_sync(kFull, r1[y], 1);
        float Ln = __shfl_up_sync(kFull, r1[y + 1], 1);
        float Ls = __shfl_up_sync(kFull, r1[y - 1], 1);
        float e4 = (r1[y] + Lc) + (r0[y + 1] + r0[y - 1]);
        float d4 = (r1[y + 1] + Ln) + (r1[y - 1] + Ls);
        float v = fmaf(0.5f, e4, fmaf(0.25f, d4, r0[y]));
        int J = (t.gy0 + y) >> 1;
        if (colown && (unsigned)(y - t.HY) < (unsigned)kWOY && I < Nc && J < Nc) gc[(size_t)J * Pc + I] = v;
    }
}

template <int OP>
__device__ __forceinline__ void wdown(const WTile &t, const float *__restrict__ g, float *__restrict__ e_out,
                                      float *__restrict__ gc, int Pc, int nu, float beta) {
    float e0[kWH], e1[kWH], g0[kWH], g1[kWH];
    wload(t, g, g0, g1);
#pragma unroll
    for (int y = 0; y < kWH; ++y) e0[y] = e1[y] = 0.f;
    wsmooth<OP>(t, e0, e1, g0, g1, nu, beta);
    wstore(t, e0, e1, e_out);
    // residual rho = (Gauss-Seidel value) - e in place of g, zero off the interior
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y) {
        float V1 = e1[y + 1] + e1[y - 1], V0 = e0[y + 1] + e0[y - 1];
        float Vl = __shfl_up_sync(kFull, V1, 1), Vr = __shfl_down_sync(kFull, V0, 1);
        float W = __shfl_up_sync(kFull, e1[y], 1), E = __shfl_down_sync(kFull, e0[y], 1);
        float ga, gb;
        if (OP == 1) {
            ga = fmaf(0.2f, (e1[y] + W) + (e0[y + 1] + e0[y - 1]), fmaf(0.05f, V1 + Vl, g0[y]));
            gb = fmaf(0.2f, (E + e0[y]) + (e1[y + 1] + e1[y - 1]), fmaf(0.05f, Vr + V0, g1[y]));
        } else {
            ga = fmaf(0.25f, (e1[y] + W) + (e0[y + 1] + e0[y - 1]), g0[y]);
            gb = fmaf(0.25f, (E + e0[y]) + (e1[y + 1] + e1[y - 1]), g1[y]);
        }
        bool rowin = t.gy0 + y >= 1 && t.gy0 + y <= t.N - 1;
        g0[y] = rowin && t.in0 ? ga - e0[y] : 0.f;
        g1[y] = rowin && t.in1 ? gb - e1[y] : 0.f;
    }
    g0[0] = g1[0] = g0[kWH - 1] = g1[kWH - 1] = 0.f;
    if (t.gy0 & 1)
        wrestrict<OP, 1>(t, g0, g1, gc, Pc);
    else
        wrestrict<OP, 0>(t, g0, g1, gc, Pc);
}

// Prolongation of the coarse correction (bilinear) added to e at the
// interior nodes of the frame, with the arithmetic of k_prolong_correct.
template <int GYP>
__device__ __forceinline__ void wprolong(const WTile &t, float (&e0)[kWH], float (&e1)[kWH],
                                         const float *__restrict__ ec, int Pc) {
    constexpr int KC = kWH / 2 + 1;  // coarse rows under the frame
    int Nc = t.N / 2;
    int I = (t.gx0 + 2 * t.lane) >> 1, J0 = t.gy0 >> 1;
    bool okI = I >= 0 && I <= Nc, okI1 = I + 1 >= 0 && I + 1 <= Nc;
    float ca[KC], cb[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        int J = J0 + k;
        bool okJ = J >= 0 && J <= Nc;
        ca[k] = okJ && okI ? __ldg(ec + (size_t)J * Pc + I) : 0.f;
        cb[k] = okJ && okI1 ? __ldg(ec + (size_t)J * Pc + I + 1) : 0.f;
    }
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y) {
        int gj = t.gy0 + y;
        if (gj < 1 || gj > t.N - 1) continue;
        int k = (y + GYP) >> 1;
        if (((y + GYP) & 1) == 0) {  // even global row
            if (t.in0) e0[y] = __fadd_rn(e0[y], ca[k]);
            if (t.in1) e1[y] = __fadd_rn(e1[y], __fmul_rn(0.5f, ca[k] + cb[k]));
        } else {
            if (t.in0) e0[y] = __fadd_rn(e0[y], __fmul_rn(0.5f, ca[k] + ca[k + 1]));
            if (t.in1) e1[y] = __fadd_rn(e1[y], __fmul_rn(0.25f, (ca[k] + cb[k]) + (ca[k + 1] + cb[k + 1])));
        }
    }
}

// Prolongation + post-smoothing: k_up's work for one warp tile.  With
// cor.psi64 set the smoothed correction is added to the FP64 solution
// (psi64 += e) instead of being stored.
template <int OP>
__device__ __forceinline__ void wup(const WTile &t, const float *__restrict__ e_in, const float *__restrict__ g,
                                    const float *__restrict__ ec, int Pc, float *__restrict__ e_out, int nu,
                                    float beta, Correct64 cor) {
    float e0[kWH], e1[kWH], g0[kWH], g1[kWH];
    wload(t, e_in, e0, e1);
    if (t.gy0 & 1)
        wprolong<1>(t, e0, e1, ec, Pc);
    else
        wprolong<0>(t, e0, e1, ec, Pc);
    wload(t, g, g0, g1);
    wsmooth<OP>(t, e0, e1, g0, g1, nu, beta);
    if (!cor.psi64) {
        wstore(t, e0, e1, e_out);
        return;
    }
    int x0 = 2 * t.lane, i0 = t.gx0 + x0;
    bool o0 = t.in0 && x0 >= t.HX && x0 < t.HX + kWOX, o1 = t.in1 && x0 + 1 >= t.HX && x0 + 1 < t.HX + kWOX;
#pragma unroll
    for (int y = 1; y < kWH - 1; ++y) {
        if (!(t.rows >> y & 1u) || (unsigned)(y - t.HY) >= (unsigned)kWOY) continue;
        int gj = t.gy0 + y;
        double *row = cor.psi64 + (size_t)gj * cor.P64;
        if (o0) {
            double p = row[i0] + f32_to_f64(e0[y]);
            row[i0] = p;
            if (cor.psi32) cor.psi32[(size_t)gj * cor.P32 + i0] = f64_to_f32(p);
        }
        if (o1) {
            double p = row[i0 + 1] + f32_to_f64(e1[y]);
            row[i0 + 1] = p;
            if (cor.psi32) cor.psi32[(size_t)gj * cor.P32 + i0 + 1] = f64_to_f32(p);
        }
    }
}

__device__ __forceinline__ bool wtile_of(int N, int local_tile, int &tx, int &ty) {
    int ntx = (N - 1 + kWOX - 1) / kWOX, nty = (N - 1 + kWOY - 1) / kWOY;
    if (local_tile >= ntx * nty) return false;
    tx = local_tile % ntx;
    ty = local_tile / ntx;
    return true;
}

template <int OP>
__global__ void __launch_bounds__(32 * kWarps)
    k_down_w(const float *__restrict__ g, float *__restrict__ e_out, int N, int P, float *__restrict__ gc, int Pc,
             int nu, float beta) {
    pdl_enter();
    int tx, ty;
    if (!wtile_of(N, blockIdx.x * kWarps + (threadIdx.x >> 5), tx, ty)) return;  // whole warps leave
    wdown<OP>(wtile(N, P, tx, ty, OP, nu), g, e_out, gc, Pc, nu, beta);
}

template <int OP>
__global__ void __launch_bounds__(32 * kWarps)
    k_up_w(const float *__restrict__ e_in, const float *__restrict__ g, const float *__restrict__ ec, int Pc,
           float *__restrict__ e_out, int N, int P, int nu, float beta, Correct64 cor) {
    pdl_enter();
    int tx, ty;
    if (!wtile_of(N, blockIdx.x * kWarps + (threadIdx.x >> 5), tx, ty)) return;
    wup<OP>(wtile(N, P, tx, ty, OP, nu), e_in, g, ec, Pc, e_out, nu, beta, cor);
}

// Batched forms: the block range table gives each cavity ceil(tiles / 4)
// blocks and its tiles per row (gx).
__device__ __forceinline__ int wlocate(const BatchRange *r, int &local) {
    int b = blockIdx.x, lo = 0, hi = r->count;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (r->start[mid] <= b) lo = mid;
        else hi = mid;
    }
    local = b - r->start[lo];
    return lo;
}

template <int OP>
__global__ void __launch_bounds__(32 * kWarps)
    k_down_w_batch(BatchCav *cav, const BatchRange *r, int level, int nu, float beta) {
    pdl_enter();
    int local;
    const BatchCav &cv = cav[wlocate(r, local)];
    if (!cv.active) return;
    int N = cv.N >> level, tx, ty;
    if (!wtile_of(N, local * kWarps + (threadIdx.x >> 5), tx, ty)) return;
    wdown<OP>(wtile(N, cv.P[level], tx, ty, OP, nu), cv.g32[level], cv.eB[level], cv.g32[level + 1], cv.P[level + 1],
              nu, beta);
}

template <int OP>
__global__ void __launch_bounds__(32 * kWarps)
    k_up_w_batch(BatchCav *cav, const BatchRange *r, int level, int nu, float beta) {
    pdl_enter();
    int local;
    const BatchCav &cv = cav[wlocate(r, local)];
    if (!cv.active) return;
    int N = cv.N >> level, tx, ty;
    if (!wtile_of(N, local * kWarps + (threadIdx.x >> 5), tx, ty)) return;
    Correct64 cor{nullptr, 0, nullptr, 0};
    if (level == 0) cor = Correct64{cv.psi64, cv.P[0], nullptr, cv.P[0]};
    wup<OP>(wtile(N, cv.P[level], tx, ty, OP, nu), cv.eB[level], cv.g32[level], cv.eA[level + 1], cv.P[level + 1],
            cv.eA[level], nu, beta, cor);
}

}  // namespace

bool warp_tile_fits(int op, int nu) { return warp_fits(op, nu); }
int warp_tile_blocks(int N) {
    int nt = ((N - 1 + kWOX - 1) / kWOX) * ((N - 1 + kWOY - 1) / kWOY);
    return (nt + kWarps - 1) / kWarps;
}

cudaError_t launch_down_warp(cudaStream_t s, int op, const float *g, float *e_out, int N, int P, float *gc, int Pc,
                             int nu, float beta) {
    if (op == 1)
        (void)launch_pdl(k_down_w<1>, warp_tile_blocks(N), 32 * kWarps, 0, s, g, e_out, N, P, gc, Pc, nu, beta);
    else
        (void)launch_pdl(k_down_w<0>, warp_tile_blocks(N), 32 * kWarps, 0, s, g, e_out, N, P, gc, Pc, nu, beta);
    return cudaGetLastError();
}

cudaError_t launch_up_warp(cudaStream_t s, int op, const float *e_in, const float *g, const float *ec, int Pc,
                           float *e_out, int N, int P, int nu, float beta, Correct64 cor) {
    if (op == 1)
        (void)launch_pdl(k_up_w<1>, warp_tile_blocks(N), 32 * kWarps, 0, s, e_in, g, ec, Pc, e_out, N, P, nu, beta,
                         cor);
    else
        (void)launch_pdl(k_up_w<0>, warp_tile_blocks(N), 32 * kWarps, 0, s, e_in, g, ec, Pc, e_out, N, P, nu, beta,
                         cor);
    return cudaGetLastError();
}

cudaError_t launch_down_warp_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, int level, int nblocks,
                                   int nu, float beta) {
    if (op == 1)
        (void)launch_pdl(k_down_w_batch<1>, nblocks, 32 * kWarps, 0, s, cav, r, level, nu, beta);
    else
        (void)launch_pdl(k_down_w_batch<0>, nblocks, 32 * kWarps, 0, s, cav, r, level, nu, beta);
    return cudaGetLastError();
}

cudaError_t launch_up_warp_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, int level, int nblocks,
                                 int nu, float beta) {
    if (op == 1)
        (void)launch_pdl(k_up_w_batch<1>, nblocks, 32 * kWarps, 0, s, cav, r, level, nu, beta);
    else
        (void)launch_pdl(k_up_w_batch<0>, nblocks, 32 * kWarps, 0, s, cav, r, level, nu, beta);
    return cudaGetLastError();
}

}  // namespace lcx
