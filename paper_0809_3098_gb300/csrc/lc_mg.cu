// Multigrid kernels that fuse a level's colour phases in shared memory.
//
// The smoother is the SOR update of Eq. (15) (Cardoso & Bicudo,
// arXiv:0809.3098, Sec. 3) in colour order; these kernels compute exactly the
// values the one-phase-per-launch kernels of lc_kernels.cu compute (same
// expression per node, same order), with fewer launches:
//
//  k_down:   load a tile of psi and g with a halo, nu1 colour sweeps, write the
//            tile's own psi, residual, full weighting onto the coarse grid;
//  k_up:     load a tile of psi plus the bilinear prolongation of the coarse
//            correction, nu2 colour sweeps, write the tile's own psi and (on
//            the fine level) the tile's sum of squared residuals;
//  k_coarse: a whole V-cycle of the coarsest levels in one block, every level
//            held in shared memory;
//  k_coarse_cluster: the same V-cycle from a larger level down, its larger
//            levels split by rows over the blocks of a thread-block cluster
//            (distributed shared memory, a cluster barrier per phase).
//
// A tile owns an aligned block of TX x TY interior nodes and recomputes a halo
// around it.  Invalid values enter a tile from its edge and spread one
// neighbour per colour phase; with the colour orders used here the residual
// after nu sweeps is exact at distances >= (4 nu + 1, 2 nu + 1) from the edge
// for the compact operator and 2 nu + 1 for the 5-point one, which sets the
// halo.  Tiles read psi from one buffer and write another (ping-pong), so no
// tile ever sees a neighbour's half-updated values.
#include "lc_internal.h"

#include <cooperative_groups.h>

#include <atomic>
#include <cmath>

namespace lcx {

namespace {

template <typename T, int OP>
__device__ __forceinline__ T gs_local(const T *sp, const T *sg, int c, int LP) {
    T n4 = (sp[c + 1] + sp[c - 1]) + (sp[c + LP] + sp[c - LP]);
    if (OP == 1) {
        T d4 = (sp[c + LP + 1] + sp[c - LP + 1]) + (sp[c + LP - 1] + sp[c - LP - 1]);
        return fma(T(0.2), n4, fma(T(0.05), d4, sg[c]));
    }
    return fma(T(0.25), n4, sg[c]);
}

// Halo (x, y) a tile needs for a valid residual after nu sweeps.
__host__ __device__ inline int halo_x(int op, int nu) { return op == 1 ? 4 * nu + 1 : 2 * nu + 1; }
__host__ __device__ inline int halo_y(int op, int nu) { return 2 * nu + 1; }
// Shared-memory tile geometry: LX x LY nodes, row pitch LP even and at least
// LX + 1 (the pair loads of the last column read one element past it).
__host__ __device__ inline int tile_lx(int TX, int op, int nu) { return TX + 2 * halo_x(op, nu) + 1; }
__host__ __device__ inline int tile_ly(int TY, int nu) { return TY + 2 * halo_y(0, nu) + 1; }
__host__ __device__ inline int tile_lp(int LX) { return (LX + 2) & ~1; }
// Coarse tile staged by k_up: the coarse nodes under LX x LY fine nodes.
__host__ __device__ inline int tile_lxc(int LX) { return LX / 2 + 3; }

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    typedef float2 type;
};
template <>
struct Pair<double> {
    typedef double2 type;
};

// W, P, E of local column x in one shared-memory row, read as two aligned
// pairs (even offsets) so that the threads of a warp, which take every other
// column, read contiguous memory without bank conflicts.
template <typename T>
__device__ __forceinline__ void row3(const T *row, int x, bool xodd, T &w, T &p, T &e) {
    typedef typename Pair<T>::type P2;
    if (xodd) {
        P2 a = *reinterpret_cast<const P2 *>(row + x - 1), b = *reinterpret_cast<const P2 *>(row + x + 1);
        w = a.x;
        p = a.y;
        e = b.x;
    } else {
        P2 a = *reinterpret_cast<const P2 *>(row + x - 2), b = *reinterpret_cast<const P2 *>(row + x);
        w = a.y;
        p = b.x;
        e = b.y;
    }
}

template <typename T>
__device__ __forceinline__ T mid1(const T *row, int x, bool xodd) {
    typedef typename Pair<T>::type P2;
    return xodd ? reinterpret_cast<const P2 *>(row + x - 1)->y : reinterpret_cast<const P2 *>(row + x)->x;
}

// Gauss-Seidel value of node (x, y) from pair loads; the operand order is the
// one of gs_local, so the result is bit-identical.
template <typename T, int OP>
__device__ __forceinline__ T gs_pairs(const T *sp, const T *sg, int LP, int x, int y, bool xodd, T &pc) {
    const T *r0 = sp + y * LP;
    T w, p, e;
    row3<T>(r0, x, xodd, w, p, e);
    pc = p;
    if (OP == 1) {
        T nw, n, ne, sw, so, se;
        row3<T>(r0 + LP, x, xodd, nw, n, ne);
        row3<T>(r0 - LP, x, xodd, sw, so, se);
        T n4 = (e + w) + (n + so);
        T d4 = (ne + se) + (nw + sw);
        return fma(T(0.2), n4, fma(T(0.05), d4, sg[y * LP + x]));
    }
    T n = mid1<T>(r0 + LP, x, xodd), so = mid1<T>(r0 - LP, x, xodd);
    T n4 = (e + w) + (n + so);
    return fma(T(0.25), n4, sg[y * LP + x]);
}

// Updates a pair of same-colour nodes (x, y) and (x, y + 2) from pair loads:
// rows y - 1 .. y + 3, row y + 1 shared; same operands and order as gs_local.
template <typename T, int OP>
__device__ __forceinline__ void update_pair(T *sp, const T *sg, int LP, int x, int y, bool xodd, bool two, T beta) {
    T *r0 = sp + y * LP;
    T aw, ap, ae, bw, bp, be, cw, cp, ce;  // rows y - 1, y, y + 1
    row3<T>(r0 - LP, x, xodd, aw, ap, ae);
    row3<T>(r0, x, xodd, bw, bp, be);
    row3<T>(r0 + LP, x, xodd, cw, cp, ce);
    T v1;
    if (OP == 1) {
        T n4 = (be + bw) + (cp + ap);
        T d4 = (ce + ae) + (cw + aw);
        v1 = fma(T(0.2), n4, fma(T(0.05), d4, sg[y * LP + x]));
    } else {
        v1 = fma(T(0.25), (be + bw) + (cp + ap), sg[y * LP + x]);
    }
    if (beta != T(1)) v1 = fma(beta, v1 - bp, bp);
    if (two) {
        T dw, dp, de, ew, ep, ee;  // rows y + 2, y + 3
        row3<T>(r0 + 2 * LP, x, xodd, dw, dp, de);
        row3<T>(r0 + 3 * LP, x, xodd, ew, ep, ee);
        T v2;
        if (OP == 1) {
            T n4 = (de + dw) + (ep + cp);
            T d4 = (ee + ce) + (ew + cw);
            v2 = fma(T(0.2), n4, fma(T(0.05), d4, sg[(y + 2) * LP + x]));
        } else {
            v2 = fma(T(0.25), (de + dw) + (ep + cp), sg[(y + 2) * LP + x]);
        }
        if (beta != T(1)) v2 = fma(beta, v2 - dp, dp);
        r0[2 * LP + x] = v2;
    }
    r0[x] = v1;
}

// One colour phase over the tile's updatable nodes: local [1, LX-2] x
// [1, LY-2] intersected with the domain interior ([xlo, xhi] x [ylo, yhi]).
// Block is 2-D with blockDim.x = 32; each thread updates two nodes of the
// colour in one column (rows y and y + 2).
template <typename T, int OP>
__device__ void tile_phase(T *sp, const T *sg, int LP, int xlo, int xhi, int ylo, int yhi, int gx0, int gy0,
                           int colour, T beta) {
    if (OP == 1) {
        int pi = colour & 1, pj = colour >> 1;
        int x0 = ((gx0 + xlo) & 1) == pi ? xlo : xlo + 1;  // first column of the colour
        int y0 = ((gy0 + ylo) & 1) == pj ? ylo : ylo + 1;
        bool xodd = x0 & 1;
        for (int y = y0 + 4 * (int)threadIdx.y; y <= yhi; y += 4 * blockDim.y) {
            bool two = y + 2 <= yhi;
            for (int x = x0 + 2 * (int)threadIdx.x; x <= xhi; x += 2 * blockDim.x)
                update_pair<T, OP>(sp, sg, LP, x, y, xodd, two, beta);
        }
    } else {
        // rows y and y + 2 share a parity: thread rows (ylo, ylo+2), (ylo+1, ylo+3), (ylo+4, ...)
        for (int k = threadIdx.y; ; k += blockDim.y) {
            int y = ylo + 4 * (k >> 1) + (k & 1);
            if (y > yhi) break;
            bool two = y + 2 <= yhi;
            int x0 = ((gx0 + xlo + gy0 + y) & 1) == colour ? xlo : xlo + 1;
            bool xodd = x0 & 1;
            for (int x = x0 + 2 * (int)threadIdx.x; x <= xhi; x += 2 * blockDim.x)
                update_pair<T, OP>(sp, sg, LP, x, y, xodd, two, beta);
        }
    }
}

template <typename T, int OP>
__device__ void tile_sweeps(T *sp, const T *sg, int LP, int LX, int LY, int gx0, int gy0, int N, int nu, T beta) {
    int ncol = OP == 1 ? 4 : 2;
    // updatable local range: [1, L-2] and the domain interior [1, N-1]
    int xlo = max(1, 1 - gx0), xhi = min(LX - 2, N - 1 - gx0);
    int ylo = max(1, 1 - gy0), yhi = min(LY - 2, N - 1 - gy0);
    for (int s = 0; s < nu; ++s)
        for (int col = 0; col < ncol; ++col) {
            tile_phase<T, OP>(sp, sg, LP, xlo, xhi, ylo, yhi, gx0, gy0, col, beta);
            __syncthreads();
        }
}

// Asynchronous global -> shared copy of one element; an invalid element is
// filled with zero (source size 0: nothing is read from src).
template <typename T>
__device__ __forceinline__ void cp_async_el(T *dst, const T *src, bool valid) {
    unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    int n = valid ? (int)sizeof(T) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ double block_sum2d(double v, double *sh) {
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

// ---------------------------------------------------------------------------
// Pre-smoothing + residual + full weighting.  Owner region of block (bx, by):
// fine nodes [1 + bx TX, 1 + (bx+1) TX) x [1 + by TY, ...); it computes the
// coarse nodes I with 2I inside that range.  zero_init: psi starts at 0 (the
// coarse-level correction), psi_in is not read.
template <typename T, int OP, int TX, int TY>
__device__ __forceinline__ void down_body(int bx, int by, const T *__restrict__ psi_in, int zero_init,
                                          const T *__restrict__ g, T *__restrict__ psi_out, int N, int P,
                                          T *__restrict__ gc, int Pc, int nu, T beta, unsigned char *smem_raw) {
    T *sp = reinterpret_cast<T *>(smem_raw);
    int RX = halo_x(OP, nu), RY = halo_y(OP, nu);
    int LX = tile_lx(TX, OP, nu), LY = tile_ly(TY, nu), LP = tile_lp(LX);
    T *sg = sp + LY * LP;
    int ox0 = 1 + bx * TX, oy0 = 1 + by * TY;
    int gx0 = ox0 - RX, gy0 = oy0 - RY;
    for (int y = threadIdx.y; y < LY; y += blockDim.y) {
        int gj = gy0 + y;
        bool rowok = gj >= 0 && gj <= N;
        for (int x = threadIdx.x; x < LP; x += blockDim.x) {
            int gi = gx0 + x;
            bool ok = rowok && gi >= 0 && gi <= N && x < LX;
            size_t c = ok ? (size_t)gj * P + gi : 0;
            cp_async_el<T>(sg + y * LP + x, g + c, ok);
            if (zero_init)
                sp[y * LP + x] = T(0);
            else
                cp_async_el<T>(sp + y * LP + x, psi_in + c, ok);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    tile_sweeps<T, OP>(sp, sg, LP, LX, LY, gx0, gy0, N, nu, beta);
    // own psi out; residual (in place of g) on the owner region plus one node
    for (int y = RY + threadIdx.y; y <= RY + TY; y += blockDim.y) {
        int gj = gy0 + y;
        for (int x = RX + threadIdx.x; x <= RX + TX; x += blockDim.x) {
            int gi = gx0 + x;
            int c = y * LP + x;
            bool interior = gi >= 1 && gi < N && gj >= 1 && gj < N;
            if (interior && x < RX + TX && y < RY + TY) psi_out[(size_t)gj * P + gi] = sp[c];
            sg[c] = interior ? rho_node<T, OP>(sp, sg, c, LP) : T(0);
        }
    }
    __syncthreads();
    // full weighting: g_c = 4 R(rho)
    int Nc = N / 2;
    int I0 = (ox0 + 1) / 2, J0 = (oy0 + 1) / 2;
    for (int J = J0 + threadIdx.y; J < J0 + TY / 2; J += blockDim.y) {
        if (J >= Nc) break;
        for (int I = I0 + threadIdx.x; I < I0 + TX / 2; I += blockDim.x) {
            if (I >= Nc) break;
            int x = 2 * I - gx0, y = 2 * J - gy0;
            const T *r = sg + y * LP + x;
            T e4 = (r[1] + r[-1]) + (r[LP] + r[-LP]);
            T d4 = (r[LP + 1] + r[LP - 1]) + (r[-LP + 1] + r[-LP - 1]);
            gc[(size_t)J * Pc + I] = fma(T(0.5), e4, fma(T(0.25), d4, r[0]));
        }
    }
}

template <typename T, int OP, int TX, int TY>
__global__ void __launch_bounds__(512)
    k_down(const T *__restrict__ psi_in, int zero_init, const T *__restrict__ g, T *__restrict__ psi_out, int N,
           int P, T *__restrict__ gc, int Pc, int nu, T beta) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    down_body<T, OP, TX, TY>(blockIdx.x, blockIdx.y, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta, smem_raw);
}

// Prolongation + correction + post-smoothing; on the fine level also the
// tile's sum of rho^2 over its owner nodes (partials != nullptr).  With
// cor.psi64 set (the mixed-precision fine level) the smoothed correction is
// not stored: it is added to the FP64 solution, psi64 += e, and the FP32
// shadow of the new psi64 is written.  The coarse correction under the tile
// is staged in shared memory first.
template <typename T, int OP, int TX, int TY>
__device__ __forceinline__ double up_body(int bx, int by, const T *__restrict__ psi_in, const T *__restrict__ g,
                                          const T *__restrict__ ec, int Pc, T *__restrict__ psi_out, int N, int P,
                                          int nu, T beta, bool want_norm, Correct64 cor, unsigned char *smem_raw) {
    T *sp = reinterpret_cast<T *>(smem_raw);
    int RX = halo_x(OP, nu), RY = halo_y(OP, nu);
    int LX = tile_lx(TX, OP, nu), LY = tile_ly(TY, nu), LP = tile_lp(LX);
    int LXc = tile_lxc(LX), LYc = tile_lxc(LY);
    T *sg = sp + LY * LP, *sc = sg + LY * LP;
    int ox0 = 1 + bx * TX, oy0 = 1 + by * TY;
    int gx0 = ox0 - RX, gy0 = oy0 - RY;
    int Ic0 = gx0 >> 1, Jc0 = gy0 >> 1, Nc = N / 2;  // floor, also for negative gx0
    for (int y = threadIdx.y; y < LY; y += blockDim.y) {
        int gj = gy0 + y;
        bool rowok = gj >= 0 && gj <= N;
        for (int x = threadIdx.x; x < LP; x += blockDim.x) {
            int gi = gx0 + x;
            bool ok = rowok && gi >= 0 && gi <= N && x < LX;
            size_t c = ok ? (size_t)gj * P + gi : 0;
            cp_async_el<T>(sp + y * LP + x, psi_in + c, ok);
            cp_async_el<T>(sg + y * LP + x, g + c, ok);
        }
    }
    for (int Y = threadIdx.y; Y < LYc; Y += blockDim.y) {
        int J = Jc0 + Y;
        for (int X = threadIdx.x; X < LXc; X += blockDim.x) {
            int I = Ic0 + X;
            bool ok = J >= 0 && J <= Nc && I >= 0 && I <= Nc;
            cp_async_el<T>(sc + Y * LXc + X, ec + (ok ? (size_t)J * Pc + I : 0), ok);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    for (int y = threadIdx.y; y < LY; y += blockDim.y) {
        int gj = gy0 + y;
        if (gj < 1 || gj >= N) continue;
        for (int x = threadIdx.x; x < LX; x += blockDim.x) {
            int gi = gx0 + x;
            if (gi < 1 || gi >= N) continue;
            int cc = ((gj >> 1) - Jc0) * LXc + ((gi >> 1) - Ic0);
            T e;
            if (!(gi & 1) && !(gj & 1))
                e = sc[cc];
            else if ((gi & 1) && !(gj & 1))
                e = mul_rn(T(0.5), sc[cc] + sc[cc + 1]);
            else if (!(gi & 1) && (gj & 1))
                e = mul_rn(T(0.5), sc[cc] + sc[cc + LXc]);
            else
                e = mul_rn(T(0.25), (sc[cc] + sc[cc + 1]) + (sc[cc + LXc] + sc[cc + LXc + 1]));
            sp[y * LP + x] = add_rn(sp[y * LP + x], e);
        }
    }
    __syncthreads();
    tile_sweeps<T, OP>(sp, sg, LP, LX, LY, gx0, gy0, N, nu, beta);
    double acc = 0.0;
    for (int y = RY + threadIdx.y; y < RY + TY; y += blockDim.y) {
        int gj = gy0 + y;
        if (gj >= N) break;
        for (int x = RX + threadIdx.x; x < RX + TX; x += blockDim.x) {
            int gi = gx0 + x;
            if (gi >= N) break;
            int c = y * LP + x;
            if (cor.psi64) {
                size_t c64 = (size_t)gj * cor.P64 + gi;
                double pnew = cor.psi64[c64] + to_f64<T>(sp[c]);
                cor.psi64[c64] = pnew;
                if (cor.psi32) cor.psi32[(size_t)gj * cor.P32 + gi] = f64_to_f32(pnew);
            } else {
                psi_out[(size_t)gj * P + gi] = sp[c];
            }
            if (want_norm) {
                double r = (double)rho_node<T, OP>(sp, sg, c, LP);
                acc += r * r;
            }
        }
    }
    return acc;  // this thread's share of the tile's sum of rho^2
}

template <typename T, int OP, int TX, int TY>
__global__ void __launch_bounds__(512)
    k_up(const T *__restrict__ psi_in, const T *__restrict__ g, const T *__restrict__ ec, int Pc,
         T *__restrict__ psi_out, int N, int P, int nu, T beta, double *__restrict__ partials, Correct64 cor,
         FinishArgs fin) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    double acc = up_body<T, OP, TX, TY>(blockIdx.x, blockIdx.y, psi_in, g, ec, Pc, psi_out, N, P, nu, beta,
                                        partials != nullptr, cor, smem_raw);
    if (partials) {
        acc = block_sum2d(acc, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = acc;
        if (fin.enabled) finish_if_last(partials, fin);
    }
}

// ---------------------------------------------------------------------------
// A V-cycle over levels N0, N0/2, ..., down to 2 or 3 intervals, in one block
// with every level in shared memory (level k: psi then g, pitch N_k + 1,
// starting at offset sum_{k'<k} 2 (N_k' + 1)^2).  g_in: right-hand side of
// the top level; psi_warm: its initial guess (nullptr = zero); psi_out: where
// the top level's result goes; partial: if set, the sum of rho^2 of the top
// level after the cycle (and the end-of-cycle decision if fin.enabled).
template <typename T, int OP>
__device__ __forceinline__ void cs_update(T *sp, const T *sg, int c, int LP, T beta) {
    T v = gs_local<T, OP>(sp, sg, c, LP);
    if (beta != T(1)) v = fma(beta, v - sp[c], sp[c]);
    sp[c] = v;
}

// FP64 loops of the one-block levels take their nodes packed into whole
// warps: on GB300 an FP64 warp instruction occupies its SM sub-partition's
// FP64 unit for about 64 clocks however few lanes are active, so a phase of a
// few dozen nodes costs (FP64 instructions per warp) x 64 clocks on the
// busiest sub-partition, and half-empty warps double it.  The nodes of a
// phase are independent, so the order of the work does not change a value.
template <typename T>
constexpr bool kPacked = sizeof(T) == 8;

template <typename T, int OP>
__device__ void cs_sweeps(T *sp, const T *sg, int n, int nu, T beta) {
    int LP = n + 1, m = n - 1;
    if constexpr (kPacked<T>) {
        const unsigned tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
        for (int s = 0; s < nu; ++s)
            for (int col = 0; col < (OP == 1 ? 4 : 2); ++col) {
                if (OP == 1) {
                    const int x0 = (col & 1) ? 1 : 2, y0 = (col >> 1) ? 1 : 2;
                    const unsigned nx = m >= x0 ? (m - x0) / 2 + 1 : 0, ny = m >= y0 ? (m - y0) / 2 + 1 : 0;
                    for (unsigned q = tid; q < nx * ny; q += nt) {
                        const unsigned yy = q / nx, xx = q - yy * nx;
                        cs_update<T, OP>(sp, sg, (y0 + 2 * (int)yy) * LP + x0 + 2 * (int)xx, LP, beta);
                    }
                } else {
                    const unsigned hx = (m + 1) / 2;  // most nodes of one colour in a row
                    for (unsigned q = tid; q < (unsigned)m * hx; q += nt) {
                        const unsigned yy = q / hx, k = q - yy * hx;
                        const int y = 1 + (int)yy, x = (((1 + y) & 1) == col ? 1 : 2) + 2 * (int)k;
                        if (x <= m) cs_update<T, OP>(sp, sg, y * LP + x, LP, beta);
                    }
                }
                __syncthreads();
            }
    } else {
        for (int s = 0; s < nu; ++s)
            for (int col = 0; col < (OP == 1 ? 4 : 2); ++col) {
                if (OP == 1) {
                    int x0 = (col & 1) ? 1 : 2, y0 = (col >> 1) ? 1 : 2;
                    for (int y = y0 + 2 * (int)threadIdx.y; y <= m; y += 2 * blockDim.y)
                        for (int x = x0 + 2 * (int)threadIdx.x; x <= m; x += 2 * blockDim.x)
                            cs_update<T, OP>(sp, sg, y * LP + x, LP, beta);
                } else {
                    for (int y = 1 + threadIdx.y; y <= m; y += blockDim.y) {
                        int x0 = ((1 + y) & 1) == col ? 1 : 2;
                        for (int x = x0 + 2 * (int)threadIdx.x; x <= m; x += 2 * blockDim.x)
                            cs_update<T, OP>(sp, sg, y * LP + x, LP, beta);
                    }
                }
                __syncthreads();
            }
    }
}

// ---------------------------------------------------------------------------
// Exact solve of the last level of a V-cycle (the coarse solve of the
// multigrid; nuc = 0 selects it).  In the scaled form the level's equation is
//     (I - 0.2 N4 - 0.05 D4) psi = g   (compact)     (I - 0.25 N4) psi = g   (5-point)
// on the m x m interior nodes (m = n - 1), with N4 / D4 the sums of the edge /
// diagonal neighbours and psi = 0 on the walls.  Both neighbour sums are
// diagonalised by the 2-D sine transform: with S[a][y] = sqrt(2/n)
// sin(pi (a+1)(y+1) / n), symmetric and its own inverse, and c_a =
// cos(pi (a+1) / n), the sine mode (a, b) has N4 = 2 c_a + 2 c_b and
// D4 = (2 c_a)(2 c_b), so
//     psi = S ((S G S) ./ lambda) S,   lambda_ab = 1 - 0.2 (2c_a + 2c_b) - 0.05 (2c_a)(2c_b)
// (5-point: 1 - 0.25 (2c_a + 2c_b)), G the interior g as rows y, columns x.
// The host computes S and W = 1 / lambda in FP64 for every level size
// 2 <= n <= kDirectMaxN, for both operators; the FP32 kernels use the same
// values rounded.  Each output of each of the four m x m products is one
// thread's FMA chain in a fixed order, so every kernel that solves a level
// this way gives the same bits.
//
// The scheme is exactly equivariant under the mirror x -> 1 - x with
// psi -> -psi (lid reversal), as the smoother is: the table's rows obey
// S[m-1-x][b] = (-1)^b S[x][b] bit for bit (the host computes the first half
// and mirrors it; the middle row of an odd m holds exact zeros and +-sqrt(2/n)),
// the products along x run with x as the output index, and the one sum over
// x takes x and m-1-x as a pair, S[x][b] (A[x] +- A[m-1-x]), so a mirrored
// input gives the same terms in the same order with exact sign flips.
constexpr int kDirectMaxN = 16;
// entries of S, W (5-point) and W (compact) for n = 2 .. kDirectMaxN
constexpr int kDirectTable = 3 * (kDirectMaxN - 1) * kDirectMaxN * (2 * kDirectMaxN - 1) / 6;
// scratch of direct_level: S, W and two m x m products
constexpr int kDirectScratch = 4 * (kDirectMaxN - 1) * (kDirectMaxN - 1);

__device__ double g_direct64[kDirectTable];
__device__ float g_direct32[kDirectTable];

// Offset of level size n's block (S, W 5-point, W compact) in the tables.
__host__ __device__ constexpr int direct_off(int n) { return (n - 2) * (n - 1) * (2 * n - 3) / 2; }

template <typename T>
__device__ __forceinline__ const T *direct_table();
template <>
__device__ __forceinline__ const double *direct_table<double>() {
    return g_direct64;
}
template <>
__device__ __forceinline__ const float *direct_table<float>() {
    return g_direct32;
}

template <typename T, int OP>
__device__ void direct_level(T *sp, const T *sg, int n, T *scr) {
    if (n < 2 || n > kDirectMaxN) return;  // the host never asks for it: the tables stop at kDirectMaxN
    const int m = n - 1, LP = n + 1, mm = m * m;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    const T *tab = direct_table<T>() + direct_off(n);
    T *S = scr, *W = scr + mm, *A = scr + 2 * mm, *B = scr + 3 * mm;
    for (int q = tid; q < mm; q += nt) {
        S[q] = tab[q];
        W[q] = tab[(OP == 1 ? 2 : 1) * mm + q];
    }
    __syncthreads();
    for (int q = tid; q < mm; q += nt) {  // A = S G (along y; x is carried)
        const int a = q / m, x = q - a * m;
        T v = T(0);
        for (int y = 0; y < m; ++y) v = fma(S[y * m + a], sg[(y + 1) * LP + x + 1], v);
        A[q] = v;
    }
    __syncthreads();
    const int half = m >> 1;
    for (int q = tid; q < mm; q += nt) {  // B = (A S) ./ lambda, the x sum in mirror pairs
        const int a = q / m, b = q - a * m;
        const T *Ar = A + a * m;
        T v = T(0);
        for (int x = 0; x < half; ++x) {
            const T p = (b & 1) ? Ar[x] - Ar[m - 1 - x] : Ar[x] + Ar[m - 1 - x];
            v = fma(S[x * m + b], p, v);
        }
        if (m & 1) v = fma(S[half * m + b], Ar[half], v);
        B[q] = v * W[q];
    }
    __syncthreads();
    for (int q = tid; q < mm; q += nt) {  // A = S B (along y)
        const int y = q / m, b = q - y * m;
        T v = T(0);
        for (int a = 0; a < m; ++a) v = fma(S[y * m + a], B[a * m + b], v);
        A[q] = v;
    }
    __syncthreads();
    for (int q = tid; q < mm; q += nt) {  // psi = A S (along x; x is the output index)
        const int y = q / m, x = q - y * m;
        T v = T(0);
        for (int b = 0; b < m; ++b) v = fma(A[y * m + b], S[x * m + b], v);
        sp[(y + 1) * LP + x + 1] = v;
    }
    __syncthreads();
}

// Full weighting of the residual sr around fine node (2X, 2Y) onto coarse
// node (X, Y); the coarse correction starts from zero.
template <typename T>
__device__ __forceinline__ void restrict_node(const T *sr, int LP, T *sgc, T *spc, int LPc, int X, int Y) {
    const T *r = sr + (2 * Y) * LP + 2 * X;
    T e4 = (r[1] + r[-1]) + (r[LP] + r[-LP]);
    T d4 = (r[LP + 1] + r[LP - 1]) + (r[-LP + 1] + r[-LP - 1]);
    sgc[Y * LPc + X] = fma(T(0.5), e4, fma(T(0.25), d4, r[0]));
    spc[Y * LPc + X] = T(0);
}

// Bilinear prolongation of the coarse correction ec onto fine node (i, j),
// added to psi.
template <typename T>
__device__ __forceinline__ void prolong_add(T *sp, const T *ec, int LP, int LPc, int i, int j) {
    int I = i >> 1, J = j >> 1, cc = J * LPc + I;
    T e;
    if (!(i & 1) && !(j & 1))
        e = ec[cc];
    else if ((i & 1) && !(j & 1))
        e = mul_rn(T(0.5), ec[cc] + ec[cc + 1]);
    else if (!(i & 1) && (j & 1))
        e = mul_rn(T(0.5), ec[cc] + ec[cc + LPc]);
    else
        e = mul_rn(T(0.25), (ec[cc] + ec[cc + 1]) + (ec[cc + LPc] + ec[cc + LPc + 1]));
    sp[j * LP + i] = add_rn(sp[j * LP + i], e);
}

// A V-cycle over nl levels held in shared memory from base: psi and g of each
// level ((n + 1)^2 each, n = N0 >> k), level after level, boundaries zero;
// sr is residual scratch of max((N0 + 1)^2, kDirectScratch).  psi and g of the
// top level are set on entry; the coarser levels' psi is reset here.  The
// last level gets nuc colour sweeps, or with nuc = 0 its exact solve
// (direct_level).  The whole block runs it.
template <typename T, int OP>
__device__ __forceinline__ void smem_vcycle(T *base, T *sr, int N0, int nl, int nu1, int nu2, int nuc, T beta) {
    int tx = threadIdx.x, ty = threadIdx.y, bx = blockDim.x, by = blockDim.y;
    const int tid = ty * bx + tx, nt = bx * by;
    // down
    int off = 0;
    for (int k = 0; k + 1 < nl; ++k) {
        int n = N0 >> k, LP = n + 1, nc = n / 2, LPc = nc + 1;
        T *sp = base + off, *sg = sp + LP * LP;
        T *spc = sg + LP * LP, *sgc = spc + LPc * LPc;
        cs_sweeps<T, OP>(sp, sg, n, nu1, beta);
        if constexpr (kPacked<T>) {
            const unsigned m = n - 1, mc = nc - 1;
            for (unsigned q = tid; q < m * m; q += nt) {
                const unsigned yy = q / m;
                const int c = (1 + (int)yy) * LP + 1 + (int)(q - yy * m);
                sr[c] = rho_node<T, OP>(sp, sg, c, LP);
            }
            for (int q = tid; q < 4 * n; q += nt) {  // the boundary ring
                const int side = q / n, k = q - side * n;
                sr[side == 0 ? k : side == 1 ? n * LP + k + 1 : side == 2 ? (k + 1) * LP : k * LP + n] = T(0);
            }
            __syncthreads();
            for (unsigned q = tid; q < mc * mc; q += nt) {
                const unsigned yy = q / mc;
                restrict_node<T>(sr, LP, sgc, spc, LPc, 1 + (int)(q - yy * mc), 1 + (int)yy);
            }
            __syncthreads();
        } else {
            for (int y = ty; y <= n; y += by)
                for (int x = tx; x <= n; x += bx) {
                    int q = y * LP + x;
                    sr[q] = (x >= 1 && x < n && y >= 1 && y < n) ? rho_node<T, OP>(sp, sg, q, LP) : T(0);
                }
            __syncthreads();
            for (int Y = 1 + ty; Y < nc; Y += by)
                for (int X = 1 + tx; X < nc; X += bx) restrict_node<T>(sr, LP, sgc, spc, LPc, X, Y);
            __syncthreads();
        }
        off += 2 * LP * LP;
    }
    {
        int n = N0 >> (nl - 1), LP = n + 1;
        T *sp = base + off, *sg = sp + LP * LP;
        if (nuc <= 0)
            direct_level<T, OP>(sp, sg, n, sr);
        else  // with one unknown and beta = 1 a single sweep is already exact
            cs_sweeps<T, OP>(sp, sg, n, (n == 2 && beta == T(1)) ? 1 : nuc, beta);
    }
    // up
    for (int k = nl - 2; k >= 0; --k) {
        int n = N0 >> k, LP = n + 1, LPc = n / 2 + 1;
        off -= 2 * LP * LP;
        T *sp = base + off, *sg = sp + LP * LP;
        const T *ec = sg + LP * LP;
        const unsigned m = n - 1;
        if constexpr (kPacked<T>) {
            // one (i, j) parity class after the other, so that a warp's nodes
            // take one branch of prolong_add (0-3 FP64 operations)
            for (int cls = 0; cls < 4; ++cls) {
                const int i0 = 1 + (cls & 1), j0 = 1 + (cls >> 1);
                const unsigned nx = m >= (unsigned)i0 ? (m - i0) / 2 + 1 : 0;
                const unsigned ny = m >= (unsigned)j0 ? (m - j0) / 2 + 1 : 0;
                for (unsigned q = tid; q < nx * ny; q += nt) {
                    const unsigned yy = q / nx;
                    prolong_add<T>(sp, ec, LP, LPc, i0 + 2 * (int)(q - yy * nx), j0 + 2 * (int)yy);
                }
            }
        } else {
            for (int j = 1 + ty; j < n; j += by)
                for (int i = 1 + tx; i < n; i += bx) prolong_add<T>(sp, ec, LP, LPc, i, j);
        }
        __syncthreads();
        cs_sweeps<T, OP>(sp, sg, n, nu2, beta);
    }
}

template <typename T, int OP>
__device__ __forceinline__ double coarse_body(const T *__restrict__ g_in, int Pg, const T *__restrict__ psi_warm,
                                              T *__restrict__ psi_out, int Po, int N0, int nl, int nu1, int nu2,
                                              int nuc, T beta, bool want_norm, unsigned char *smem_raw) {
    T *base = reinterpret_cast<T *>(smem_raw);
    int tx = threadIdx.x, ty = threadIdx.y, bx = blockDim.x, by = blockDim.y;
    int tid = ty * bx + tx, nt = bx * by;
    int total = 0;
    for (int k = 0; k < nl; ++k) total += 2 * ((N0 >> k) + 1) * ((N0 >> k) + 1);
    T *sr = base + total;  // residual scratch, (N0+1)^2
    for (int q = tid; q < total; q += nt) base[q] = T(0);
    __syncthreads();
    int L0 = N0 + 1;
    for (int y = 1 + ty; y < N0; y += by)
        for (int x = 1 + tx; x < N0; x += bx) {
            base[L0 * L0 + y * L0 + x] = g_in[(size_t)y * Pg + x];
            if (psi_warm) base[y * L0 + x] = psi_warm[(size_t)y * Po + x];
        }
    __syncthreads();
    smem_vcycle<T, OP>(base, sr, N0, nl, nu1, nu2, nuc, beta);
    double acc = 0.0;
    for (int y = 1 + ty; y < N0; y += by)
        for (int x = 1 + tx; x < N0; x += bx) {
            int q = y * L0 + x;
            psi_out[(size_t)y * Po + x] = base[q];
            if (want_norm) {
                double r = (double)rho_node<T, OP>(base, base + L0 * L0, q, L0);
                acc += r * r;
            }
        }
    return acc;
}

template <typename T, int OP>
__global__ void __launch_bounds__(1024)
    k_coarse(const T *__restrict__ g_in, int Pg, const T *__restrict__ psi_warm, T *__restrict__ psi_out, int Po,
             int N0, int nl, int nu1, int nu2, int nuc, T beta, double *__restrict__ partial, FinishArgs fin) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    double acc = coarse_body<T, OP>(g_in, Pg, psi_warm, psi_out, Po, N0, nl, nu1, nu2, nuc, beta, partial != nullptr,
                                    smem_raw);
    if (partial) {
        acc = block_sum2d(acc, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) partial[0] = acc;
        if (fin.enabled) finish_if_last(partial, fin);
    }
}

constexpr int kTBX = 32;
// Threads per tile block: 32 x 16 for 54-row tiles, 32 x 8 otherwise, so that
// with the compact operator and nu = 2 (halo 9 x 5) a colour phase's nodes
// (at most 64 columns x 32 rows for 110 x 54, 32 x 16 for 46 x 22) fill whole
// warps with two rows per thread.
constexpr int tile_by(int TY) { return TY >= 54 ? 16 : 8; }

// Shared memory of a tile kernel: psi and g tiles, plus k_up's coarse tile.
template <typename T, int TX, int TY>
size_t down_smem(int op, int nu) {
    int LX = tile_lx(TX, op, nu), LY = tile_ly(TY, nu), LP = tile_lp(LX);
    return (2 * (size_t)LY * LP + (size_t)tile_lxc(LX) * tile_lxc(LY)) * sizeof(T);
}

template <typename T, int OP, int TX, int TY>
cudaError_t down_t(cudaStream_t s, const T *psi_in, int zero_init, const T *g, T *psi_out, int N, int P, T *gc, int Pc,
                   int nu, T beta) {
    size_t sm = down_smem<T, TX, TY>(OP, nu);
    auto kern = k_down<T, OP, TX, TY>;
    dim3 grid((N - 1 + TX - 1) / TX, (N - 1 + TY - 1) / TY);
    (void)launch_pdl(kern, grid, dim3(kTBX, tile_by(TY)), sm, s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
    return cudaGetLastError();
}

template <typename T, int OP, int TX, int TY>
cudaError_t up_t(cudaStream_t s, const T *psi_in, const T *g, const T *ec, int Pc, T *psi_out, int N, int P, int nu,
                 T beta, double *partials, Correct64 cor, FinishArgs fin) {
    size_t sm = down_smem<T, TX, TY>(OP, nu);
    auto kern = k_up<T, OP, TX, TY>;
    dim3 grid((N - 1 + TX - 1) / TX, (N - 1 + TY - 1) / TY);
    (void)launch_pdl(kern, grid, dim3(kTBX, tile_by(TY)), sm, s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials,
                     cor, fin);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched forms (mixed precision, FP32 correction hierarchy): one launch
// covers the tiles of every cavity that still iterates; a cavity whose
// Poisson loop has stopped leaves its blocks idle.
template <int OP, int TX, int TY>
__global__ void __launch_bounds__(512)
    k_down_batch(BatchCav *cav, const BatchRange *r, int level, int nu, float beta) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int bx, by;
    const BatchCav &cv = cav[batch_locate(r, bx, by)];
    if (!cv.active) return;
    down_body<float, OP, TX, TY>(bx, by, nullptr, 1, cv.g32[level], cv.eB[level], cv.N >> level, cv.P[level],
                                 cv.g32[level + 1], cv.P[level + 1], nu, beta, smem_raw);
}

template <int OP, int TX, int TY>
__global__ void __launch_bounds__(512)
    k_up_batch(BatchCav *cav, const BatchRange *r, int level, int nu, float beta) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int bx, by;
    const BatchCav &cv = cav[batch_locate(r, bx, by)];
    if (!cv.active) return;
    Correct64 cor{nullptr, 0, nullptr, 0};
    if (level == 0) cor = Correct64{cv.psi64, cv.P[0], nullptr, cv.P[0]};
    up_body<float, OP, TX, TY>(bx, by, cv.eB[level], cv.g32[level], cv.eA[level + 1], cv.P[level + 1], cv.eA[level],
                               cv.N >> level, cv.P[level], nu, beta, false, cor, smem_raw);
}

template <int OP>
__global__ void __launch_bounds__(1024) k_coarse_batch(BatchCav *cav, int nu1, int nu2, int nuc, float beta) {
    pdl_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchCav &cv = cav[blockIdx.x];
    if (!cv.active) return;
    int lc = cv.lc;
    coarse_body<float, OP>(cv.g32[lc], cv.P[lc], nullptr, cv.eA[lc], cv.P[lc], cv.N >> lc, cv.nlev - lc, nu1, nu2, nuc,
                           beta, false, smem_raw);
}

// ---------------------------------------------------------------------------
// The coarse V-cycle on a thread-block cluster.  On GB300 one SM retires about
// two FP64 operations per clock, so a one-block V-cycle over levels of 32^2
// nodes and more is bound by a single SM's FP64 (or, in FP32, issue) rate.
// Here the levels above a threshold are split by rows over the C blocks of
// one cluster (one block per SM), with a cluster barrier between phases; the
// levels at or below the threshold run in block 0 alone (smem_vcycle).
//
// Block r's strip of a level is rows [lo, hi) of psi, g and the residual; psi
// has one halo row on each side.  A block that updates a node of its first or
// last row also writes the new value into the neighbour block's halo copy
// (distributed shared memory); same-colour nodes are never neighbours, so no
// block reads a value that is being written in the same phase, and the
// barrier's release / acquire makes the copies visible before the next one.
// Restriction and prolongation read the rows they need from whichever block
// owns them.  Every value is computed by the expression the one-block kernel
// uses for it, so both kernels give the same bits.

// Shared-memory layout of k_coarse_cluster (element offsets, the same in
// every block): the strips of the nd distributed levels (psi with its two
// halo rows, g, residual), then the one-block levels in smem_vcycle's layout
// (used by block 0), its residual scratch, and one row of zeros.
struct ClusterPlan {
    int N0, nl, nd, C;
    int psi[kMaxLevels], g[kMaxLevels], r[kMaxLevels];
    int single, sr, zero, total;
};

struct Strip {
    int lo, hi;
    bool on;
};

// Rows [lo, hi) of the interior rows [1, m] owned by block r of C: the first
// A = min(C, m) blocks take floor or ceil(m / A) rows each, the rest none.
__device__ __forceinline__ Strip strip_of(int m, int C, int r) {
    int A = min(C, m);
    if (r >= A) return Strip{0, 0, false};
    return Strip{1 + (r * m) / A, 1 + ((r + 1) * m) / A, true};
}

// The block whose strip holds interior row y (1 <= y <= m).
__device__ __forceinline__ int row_owner(int y, int m, int C) {
    int A = min(C, m);
    return (y * A + m - 1) / m - 1;
}

// One colour phase over a strip: the nodes and the order of cs_sweeps.
template <typename T, int OP>
__device__ __forceinline__ void strip_phase(T *ps, const T *gs, int n, Strip st, int col, T beta, T *up, T *dn) {
    const int LP = n + 1, m = n - 1;
    const int tx = threadIdx.x, ty = threadIdx.y, bx = blockDim.x, by = blockDim.y;
    if (OP == 1) {
        const int py = col >> 1, x0 = (col & 1) ? 1 : 2;
        const int y0 = st.lo + ((st.lo & 1) != py);
        for (int y = y0 + 2 * ty; y < st.hi; y += 2 * by) {
            T *row = ps + (y - st.lo + 1) * LP;
            const T *grow = gs + (y - st.lo) * LP;
            T *cu = y == st.lo ? up : nullptr, *cd = y == st.hi - 1 ? dn : nullptr;
            for (int x = x0 + 2 * tx; x <= m; x += 2 * bx) {
                T v = gs_local<T, OP>(row, grow, x, LP);
                if (beta != T(1)) v = fma(beta, v - row[x], row[x]);
                row[x] = v;
                if (cu) cu[x] = v;
                if (cd) cd[x] = v;
            }
        }
    } else {
        for (int y = st.lo + ty; y < st.hi; y += by) {
            T *row = ps + (y - st.lo + 1) * LP;
            const T *grow = gs + (y - st.lo) * LP;
            T *cu = y == st.lo ? up : nullptr, *cd = y == st.hi - 1 ? dn : nullptr;
            const int x0 = ((1 + y) & 1) == col ? 1 : 2;
            for (int x = x0 + 2 * tx; x <= m; x += 2 * bx) {
                T v = gs_local<T, OP>(row, grow, x, LP);
                if (beta != T(1)) v = fma(beta, v - row[x], row[x]);
                row[x] = v;
                if (cu) cu[x] = v;
                if (cd) cd[x] = v;
            }
        }
    }
}

template <typename T, int OP>
__global__ void __launch_bounds__(512)
    k_coarse_cluster(const T *__restrict__ g_in, int Pg, T *__restrict__ psi_out, int Po, int nu1, int nu2, int nuc,
                     T beta, ClusterPlan pl) {
    pdl_enter();
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int C = pl.C, rank = (int)cl.block_rank();
    const int tx = threadIdx.x, ty = threadIdx.y, bx = blockDim.x, by = blockDim.y;
    const int tid = ty * bx + tx, nt = bx * by;
    const int ncol = OP == 1 ? 4 : 2;

    for (int q = tid; q < pl.total; q += nt) sm[q] = T(0);
    __syncthreads();
    {
        const int n = pl.N0, LP = n + 1;
        const Strip st = strip_of(n - 1, C, rank);
        T *gs = sm + pl.g[0];
        if (st.on)
            for (int y = st.lo + ty; y < st.hi; y += by)
                for (int x = 1 + tx; x < n; x += bx) gs[(y - st.lo) * LP + x] = g_in[(size_t)y * Pg + x];
    }
    cl.sync();  // every block's arrays are set before any block writes a halo row

    // down: smoothing, residual and restriction on the distributed levels
    for (int k = 0; k < pl.nd; ++k) {
        const int n = pl.N0 >> k, m = n - 1, LP = n + 1;
        const int nc = n / 2, mc = nc - 1, LPc = nc + 1;
        const Strip st = strip_of(m, C, rank);
        T *ps = sm + pl.psi[k], *gs = sm + pl.g[k], *rs = sm + pl.r[k];
        T *up = nullptr, *dn = nullptr;
        if (st.on && rank > 0) {
            const Strip sa = strip_of(m, C, rank - 1);
            up = cl.map_shared_rank(ps + (sa.hi - sa.lo + 1) * LP, rank - 1);
        }
        if (st.on && strip_of(m, C, rank + 1).on) dn = cl.map_shared_rank(ps, rank + 1);
        for (int s = 0; s < nu1; ++s)
            for (int col = 0; col < ncol; ++col) {
                strip_phase<T, OP>(ps, gs, n, st, col, beta, up, dn);
                cl.sync();
            }
        if (st.on)
            for (int y = st.lo + ty; y < st.hi; y += by) {
                const T *row = ps + (y - st.lo + 1) * LP, *grow = gs + (y - st.lo) * LP;
                T *rrow = rs + (y - st.lo) * LP;
                for (int x = 1 + tx; x <= m; x += bx) rrow[x] = rho_node<T, OP>(row, grow, x, LP);
            }
        cl.sync();
        // full weighting of the residual rows 2Y - 1, 2Y, 2Y + 1 (owned by any block)
        const bool single = k + 1 == pl.nd;
        const Strip sc = single ? Strip{rank == 0 ? 1 : 0, rank == 0 ? nc : 0, rank == 0} : strip_of(mc, C, rank);
        if (sc.on) {
            T *pc = single ? sm + pl.single : sm + pl.psi[k + 1];
            T *gc = single ? pc + LPc * LPc : sm + pl.g[k + 1];
            const int yoff = single ? 0 : sc.lo;  // local row of coarse row Y in gc: Y - yoff
            if (!single)
                for (int q = tid; q < (sc.hi - sc.lo + 2) * LPc; q += nt) pc[q] = T(0);
            auto rrow = [&](int y) -> const T * {
                const int o = row_owner(y, m, C);
                return cl.map_shared_rank(rs + (y - strip_of(m, C, o).lo) * LP, o);
            };
            for (int Y = sc.lo + ty; Y < sc.hi; Y += by) {
                const T *rS = rrow(2 * Y - 1), *r0 = rrow(2 * Y), *rN = rrow(2 * Y + 1);
                for (int X = 1 + tx; X <= mc; X += bx) {
                    const int x = 2 * X;
                    T e4 = (r0[x + 1] + r0[x - 1]) + (rN[x] + rS[x]);
                    T d4 = (rN[x + 1] + rN[x - 1]) + (rS[x + 1] + rS[x - 1]);
                    gc[(Y - yoff) * LPc + X] = fma(T(0.5), e4, fma(T(0.25), d4, r0[x]));
                    if (single) pc[Y * LPc + X] = T(0);
                }
            }
        }
        cl.sync();
    }

    // the levels at or below the threshold, in block 0
    if (rank == 0)
        smem_vcycle<T, OP>(sm + pl.single, sm + pl.sr, pl.N0 >> pl.nd, pl.nl - pl.nd, nu1, nu2, nuc, beta);
    cl.sync();

    // up: prolongation of the coarser level's correction, then smoothing
    for (int k = pl.nd - 1; k >= 0; --k) {
        const int n = pl.N0 >> k, m = n - 1, LP = n + 1;
        const int nc = n / 2, mc = nc - 1, LPc = nc + 1;
        const Strip st = strip_of(m, C, rank);
        const bool single = k + 1 == pl.nd;
        T *ps = sm + pl.psi[k], *gs = sm + pl.g[k];
        if (st.on) {
            // own rows and both halo rows (the owners add the same correction
            // to the same value, so the copies stay equal)
            const int ylo = max(1, st.lo - 1), yhi = min(m, st.hi);
            auto crow = [&](int J) -> const T * {
                if (single) return cl.map_shared_rank(sm + pl.single + J * LPc, 0);
                if (J == 0 || J == nc) return sm + pl.zero;
                const int o = row_owner(J, mc, C);
                return cl.map_shared_rank(sm + pl.psi[k + 1] + (J - strip_of(mc, C, o).lo + 1) * LPc, o);
            };
            for (int j = ylo + ty; j <= yhi; j += by) {
                const T *c0 = crow(j >> 1), *c1 = crow((j >> 1) + 1);
                T *row = ps + (j - st.lo + 1) * LP;
                // odd columns, then even ones: the lanes of a warp share one
                // (i, j) parity and so one branch
                for (int p = 1; p <= 2; ++p)
                    for (int i = p + 2 * tx; i <= m; i += 2 * bx) {
                        const int I = i >> 1;
                        T e;
                        if (!(i & 1) && !(j & 1))
                            e = c0[I];
                        else if ((i & 1) && !(j & 1))
                            e = mul_rn(T(0.5), c0[I] + c0[I + 1]);
                        else if (!(i & 1) && (j & 1))
                            e = mul_rn(T(0.5), c0[I] + c1[I]);
                        else
                            e = mul_rn(T(0.25), (c0[I] + c0[I + 1]) + (c1[I] + c1[I + 1]));
                        row[i] = add_rn(row[i], e);
                    }
            }
        }
        cl.sync();
        T *up = nullptr, *dn = nullptr;
        if (st.on && rank > 0) {
            const Strip sa = strip_of(m, C, rank - 1);
            up = cl.map_shared_rank(ps + (sa.hi - sa.lo + 1) * LP, rank - 1);
        }
        if (st.on && strip_of(m, C, rank + 1).on) dn = cl.map_shared_rank(ps, rank + 1);
        for (int s = 0; s < nu2; ++s)
            for (int col = 0; col < ncol; ++col) {
                strip_phase<T, OP>(ps, gs, n, st, col, beta, up, dn);
                cl.sync();
            }
    }
    {
        const int n = pl.N0, LP = n + 1;
        const Strip st = strip_of(n - 1, C, rank);
        const T *ps = sm + pl.psi[0];
        if (st.on)
            for (int y = st.lo + ty; y < st.hi; y += by)
                for (int x = 1 + tx; x < n; x += bx) psi_out[(size_t)y * Po + x] = ps[(y - st.lo + 1) * LP + x];
    }
}

constexpr int kShapeTX[5] = {110, 110, 46, 16, 44};
constexpr int kShapeTY[5] = {54, 22, 22, 16, 20};
constexpr int kShapes = 5;

}  // namespace

int tile_tx(int shape) { return kShapeTX[shape]; }
int tile_ty(int shape) { return kShapeTY[shape]; }

int tiles_of(int N, int shape) {
    return ((N - 1 + kShapeTX[shape] - 1) / kShapeTX[shape]) * ((N - 1 + kShapeTY[shape] - 1) / kShapeTY[shape]);
}

size_t tile_smem_bytes(int shape, int op, int nu, int elem) {
    if (shape == 4) return elem == 4 && warp_tile_fits(op, nu) ? 0 : ~size_t(0) / 2;  // registers only
    int LX = tile_lx(kShapeTX[shape], op, nu), LY = tile_ly(kShapeTY[shape], nu), LP = tile_lp(LX);
    return (2 * (size_t)LY * LP + (size_t)tile_lxc(LX) * tile_lxc(LY)) * elem;
}

// Picks the tile shape of a level by a simple cost model.  FP64 tiles are
// bound by the SM's FP64 pipe, which the blocks resident on one SM share, so
// a launch costs (tiles per SM) x (nodes of a tile including its recomputed
// halo); FP32 tiles are latency-bound, so a launch costs (waves of resident
// blocks) x (a fixed barrier-chain latency + a small per-node term).
int tile_shape_for(int N, int op, int nu, int elem, int force) {
    if (force >= 0 && force < kShapes && tile_smem_bytes(force, op, nu, elem) <= kMaxSmem - 1024) return force;
    // The register tiles (shape 4) are only taken when forced or measured
    // faster by the batch autotuner: at 206-238 registers per thread they keep
    // 8 warps per SM, too few to hide their global loads.
    const int sms = 152;
    double best = 1e300;
    int pick = 3;
    for (int sh = 0; sh < 4; ++sh) {
        size_t sm = tile_smem_bytes(sh, op, nu, elem);
        if (sm > kMaxSmem - 1024) continue;
        int bps = (int)((kMaxSmem - 1024) / sm);
        if (bps > 4) bps = 4;
        int LX = tile_lx(kShapeTX[sh], op, nu), LY = tile_ly(kShapeTY[sh], nu);
        int nt = tiles_of(N, sh);
        double cost;
        if (elem == 8)
            cost = (double)((nt + sms - 1) / sms) * ((double)LX * LY * (nu + 1) + 1500.0);
        else
            cost = (double)((nt + sms * bps - 1) / (sms * bps)) * (0.08 * LX * LY * (nu + 1) + 3000.0);
        if (cost < best) {
            best = cost;
            pick = sh;
        }
    }
    return pick;
}

namespace {

template <typename T, int OP>
cudaError_t down_shape(cudaStream_t s, int shape, const T *psi_in, int zero_init, const T *g, T *psi_out, int N, int P,
                       T *gc, int Pc, int nu, T beta) {
    if (shape == 4) {  // FP32 register tiles, zero initial correction only
        if (sizeof(T) != 4 || !zero_init) return cudaErrorInvalidValue;
        return launch_down_warp(s, OP, reinterpret_cast<const float *>(g), reinterpret_cast<float *>(psi_out), N, P,
                                reinterpret_cast<float *>(gc), Pc, nu, (float)beta);
    }
    switch (shape) {
        case 0: return down_t<T, OP, 110, 54>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
        case 1: return down_t<T, OP, 110, 22>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
        case 2: return down_t<T, OP, 46, 22>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
        default: return down_t<T, OP, 16, 16>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
    }
}

template <typename T, int OP>
cudaError_t up_shape(cudaStream_t s, int shape, const T *psi_in, const T *g, const T *ec, int Pc, T *psi_out, int N,
                     int P, int nu, T beta, double *partials, Correct64 cor, FinishArgs fin) {
    if (shape == 4) {  // FP32 register tiles; no residual norm
        if (sizeof(T) != 4 || partials || fin.enabled) return cudaErrorInvalidValue;
        return launch_up_warp(s, OP, reinterpret_cast<const float *>(psi_in), reinterpret_cast<const float *>(g),
                              reinterpret_cast<const float *>(ec), Pc, reinterpret_cast<float *>(psi_out), N, P, nu,
                              (float)beta, cor);
    }
    switch (shape) {
        case 0: return up_t<T, OP, 110, 54>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor, fin);
        case 1: return up_t<T, OP, 110, 22>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor, fin);
        case 2: return up_t<T, OP, 46, 22>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor, fin);
        default: return up_t<T, OP, 16, 16>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor, fin);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_down(cudaStream_t s, int shape, int op, const T *psi_in, int zero_init, const T *g, T *psi_out,
                        int N, int P, T *gc, int Pc, int nu, T beta) {
    if (op == 1) return down_shape<T, 1>(s, shape, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
    return down_shape<T, 0>(s, shape, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
}

template <typename T>
cudaError_t launch_up(cudaStream_t s, int shape, int op, const T *psi_in, const T *g, const T *ec, int Pc, T *psi_out,
                      int N, int P, int nu, T beta, double *partials, Correct64 cor, FinishArgs fin) {
    if (op == 1) return up_shape<T, 1>(s, shape, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor, fin);
    return up_shape<T, 0>(s, shape, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor, fin);
}

size_t coarse_smem_bytes(int N0, int nl, int elem) {
    size_t n = 0;
    for (int k = 0; k < nl; ++k) n += 2 * (size_t)((N0 >> k) + 1) * ((N0 >> k) + 1);
    size_t sr = (size_t)(N0 + 1) * (N0 + 1);
    n += sr > (size_t)kDirectScratch ? sr : (size_t)kDirectScratch;
    return n * elem;
}

template <typename T>
cudaError_t launch_coarse(cudaStream_t s, int op, const T *g_in, int Pg, const T *psi_warm, T *psi_out, int Po, int N0,
                          int nl, int nu1, int nu2, int nuc, T beta, double *partial, FinishArgs fin) {
    size_t sm = coarse_smem_bytes(N0, nl, sizeof(T));
    auto kern = op == 1 ? k_coarse<T, 1> : k_coarse<T, 0>;
    dim3 blk(32, sizeof(T) == 8 ? 16 : 32);
    (void)launch_pdl(kern, 1, blk, sm, s, g_in, Pg, psi_warm, psi_out, Po, N0, nl, nu1, nu2, nuc, beta, partial, fin);
    return cudaGetLastError();
}

// Blocks of a cluster share one SM only if their shared memory fits it
// twice; every launch requests at least this much, so each block gets an SM
// (and its FP64 pipe) of its own.
constexpr size_t kClusterMinSmem = 120 * 1024;

static ClusterPlan cluster_plan(int N0, int nl, int C, int split) {
    ClusterPlan pl{};
    pl.N0 = N0;
    pl.nl = nl;
    pl.C = C;
    pl.nd = 0;
    while (pl.nd < nl - 1 && (N0 >> pl.nd) > split) ++pl.nd;
    int off = 0;
    auto take = [&off](int n) {
        int o = off;
        off += (n + 3) & ~3;
        return o;
    };
    for (int k = 0; k < pl.nd; ++k) {
        int n = N0 >> k, m = n - 1, A = m < C ? m : C, H = (m + A - 1) / A, LP = n + 1;
        pl.psi[k] = take((H + 2) * LP);
        pl.g[k] = take(H * LP);
        pl.r[k] = take(H * LP);
    }
    int single = 0;
    for (int k = pl.nd; k < nl; ++k) single += 2 * ((N0 >> k) + 1) * ((N0 >> k) + 1);
    pl.single = take(single);
    const int nsr = ((N0 >> pl.nd) + 1) * ((N0 >> pl.nd) + 1);
    pl.sr = take(nsr > kDirectScratch ? nsr : kDirectScratch);
    pl.zero = take(N0 + 2);
    pl.total = off;
    return pl;
}

size_t cluster_smem_bytes(int N0, int nl, int C, int split, int elem) {
    size_t b = (size_t)cluster_plan(N0, nl, C, split).total * elem;
    return b < kClusterMinSmem ? kClusterMinSmem : b;
}

template <typename T>
cudaError_t launch_coarse_cluster(cudaStream_t s, int op, const T *g_in, int Pg, T *psi_out, int Po, int N0, int nl,
                                  int nu1, int nu2, int nuc, T beta, int C, int split) {
    ClusterPlan pl = cluster_plan(N0, nl, C, split);
    size_t sm = cluster_smem_bytes(N0, nl, C, split, sizeof(T));
    if (pl.nd < 1 || C < 1 || C > 16 || sm > kMaxSmem - 1024) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(32, 16);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = tl_pdl ? 2 : 1;
    if (op == 1) return cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, 1>, g_in, Pg, psi_out, Po, nu1, nu2, nuc, beta, pl);
    return cudaLaunchKernelEx(&cfg, k_coarse_cluster<T, 0>, g_in, Pg, psi_out, Po, nu1, nu2, nuc, beta, pl);
}

// Largest cluster (16, else 8, else 0) that each device can schedule for the
// coarse cluster kernel with its largest shared memory, by device ordinal;
// found by init_mg_kernel_attributes with that device current (after the
// non-portable size is allowed).
constexpr int kMaxClusterDevices = 64;
static std::atomic<int> g_cluster_size[kMaxClusterDevices];

static int query_cluster_size() {
    for (int C : {16, 8}) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(32, 16);
        cfg.dynamicSmemBytes = kMaxSmem - 1024;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        const void *k = (const void *)k_coarse_cluster<double, 1>;
        if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n > 0) return C;
        cudaGetLastError();  // a size the device cannot schedule is not an error here
    }
    return 0;
}

int coarse_cluster_size(int device) {
    return device >= 0 && device < kMaxClusterDevices ? g_cluster_size[device].load() : 0;
}

namespace {

template <int OP, int TX, int TY>
cudaError_t down_batch_t(cudaStream_t s, BatchCav *cav, const BatchRange *r, int level, int nblocks, int nu,
                         float beta) {
    (void)launch_pdl(k_down_batch<OP, TX, TY>, nblocks, dim3(kTBX, tile_by(TY)), down_smem<float, TX, TY>(OP, nu), s,
                     cav, r, level, nu, beta);
    return cudaGetLastError();
}

template <int OP, int TX, int TY>
cudaError_t up_batch_t(cudaStream_t s, BatchCav *cav, const BatchRange *r, int level, int nblocks, int nu,
                       float beta) {
    (void)launch_pdl(k_up_batch<OP, TX, TY>, nblocks, dim3(kTBX, tile_by(TY)), down_smem<float, TX, TY>(OP, nu), s, cav,
                     r, level, nu, beta);
    return cudaGetLastError();
}

template <int OP>
cudaError_t down_batch_shape(cudaStream_t s, int shape, BatchCav *cav, const BatchRange *r, int level, int nb, int nu,
                             float beta) {
    switch (shape) {
        case 0: return down_batch_t<OP, 110, 54>(s, cav, r, level, nb, nu, beta);
        case 1: return down_batch_t<OP, 110, 22>(s, cav, r, level, nb, nu, beta);
        case 2: return down_batch_t<OP, 46, 22>(s, cav, r, level, nb, nu, beta);
        default: return down_batch_t<OP, 16, 16>(s, cav, r, level, nb, nu, beta);
    }
}

template <int OP>
cudaError_t up_batch_shape(cudaStream_t s, int shape, BatchCav *cav, const BatchRange *r, int level, int nb, int nu,
                           float beta) {
    switch (shape) {
        case 0: return up_batch_t<OP, 110, 54>(s, cav, r, level, nb, nu, beta);
        case 1: return up_batch_t<OP, 110, 22>(s, cav, r, level, nb, nu, beta);
        case 2: return up_batch_t<OP, 46, 22>(s, cav, r, level, nb, nu, beta);
        default: return up_batch_t<OP, 16, 16>(s, cav, r, level, nb, nu, beta);
    }
}

}  // namespace

template <>
cudaError_t launch_down_batch<float>(cudaStream_t s, int shape, int op, BatchCav *cav, const BatchRange *r, int level,
                                     int nblocks, int nu, float beta) {
    if (shape == 4) return launch_down_warp_batch(s, op, cav, r, level, nblocks, nu, beta);
    return op == 1 ? down_batch_shape<1>(s, shape, cav, r, level, nblocks, nu, beta)
                   : down_batch_shape<0>(s, shape, cav, r, level, nblocks, nu, beta);
}

template <>
cudaError_t launch_up_batch<float>(cudaStream_t s, int shape, int op, BatchCav *cav, const BatchRange *r, int level,
                                   int nblocks, int nu, float beta) {
    if (shape == 4) return launch_up_warp_batch(s, op, cav, r, level, nblocks, nu, beta);
    return op == 1 ? up_batch_shape<1>(s, shape, cav, r, level, nblocks, nu, beta)
                   : up_batch_shape<0>(s, shape, cav, r, level, nblocks, nu, beta);
}

cudaError_t launch_coarse_batch(cudaStream_t s, int op, BatchCav *cav, int count, int smem, int nu1, int nu2, int nuc,
                                float beta) {
    if (op == 1)
        (void)launch_pdl(k_coarse_batch<1>, count, dim3(32, 32), smem, s, cav, nu1, nu2, nuc, beta);
    else
        (void)launch_pdl(k_coarse_batch<0>, count, dim3(32, 32), smem, s, cav, nu1, nu2, nuc, beta);
    return cudaGetLastError();
}

// Raises every tile / coarse kernel's dynamic shared-memory limit once, before
// any launch or graph capture.
template <typename T>
static cudaError_t set_attrs_t() {
    const void *k[] = {
        (const void *)k_down<T, 0, 110, 54>, (const void *)k_down<T, 1, 110, 54>, (const void *)k_down<T, 0, 110, 22>,
        (const void *)k_down<T, 1, 110, 22>,  (const void *)k_down<T, 0, 46, 22>,  (const void *)k_down<T, 1, 46, 22>,
        (const void *)k_down<T, 0, 16, 16>,  (const void *)k_down<T, 1, 16, 16>,  (const void *)k_up<T, 0, 110, 54>,
        (const void *)k_up<T, 1, 110, 54>,   (const void *)k_up<T, 0, 110, 22>,    (const void *)k_up<T, 1, 110, 22>,
        (const void *)k_up<T, 0, 46, 22>,    (const void *)k_up<T, 1, 46, 22>,    (const void *)k_up<T, 0, 16, 16>,
        (const void *)k_up<T, 1, 16, 16>,    (const void *)k_coarse<T, 0>,        (const void *)k_coarse<T, 1>};
    for (const void *f : k) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxSmem - 1024));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <int OP>
static cudaError_t set_batch_attrs_t() {
    const void *k[] = {(const void *)k_down_batch<OP, 110, 54>, (const void *)k_down_batch<OP, 110, 22>,
                       (const void *)k_down_batch<OP, 46, 22>,  (const void *)k_down_batch<OP, 16, 16>,
                       (const void *)k_up_batch<OP, 110, 54>,   (const void *)k_up_batch<OP, 110, 22>,
                       (const void *)k_up_batch<OP, 46, 22>,    (const void *)k_up_batch<OP, 16, 16>,
                       (const void *)k_coarse_batch<OP>};
    for (const void *f : k) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxSmem - 1024));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename T>
static cudaError_t set_cluster_attrs_t() {
    const void *k[] = {(const void *)k_coarse_cluster<T, 0>, (const void *)k_coarse_cluster<T, 1>};
    for (const void *f : k) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxSmem - 1024));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The tables of direct_level for every level size 2 <= n <= kDirectMaxN,
// computed in FP64 on the host and copied to each device once.
static std::atomic<bool> g_direct_ready[kMaxClusterDevices];

static cudaError_t init_direct_tables(int dev) {
    if (dev < 0 || dev >= kMaxClusterDevices) return cudaErrorInvalidDevice;
    if (g_direct_ready[dev].load()) return cudaSuccess;
    static double t64[kDirectTable];
    static float t32[kDirectTable];
    const double pi = 3.14159265358979323846;
    for (int n = 2; n <= kDirectMaxN; ++n) {
        const int m = n - 1, mm = m * m;
        double *S = t64 + direct_off(n), *W5 = S + mm, *Wc = S + 2 * mm;
        const double sc = std::sqrt(2.0 / n);
        // rows x < m / 2 from the sine, the others by S[m-1-x][b] = (-1)^b S[x][b];
        // the middle row of an odd m exactly: sin(pi (b+1) / 2) is 0 or +-1
        for (int x = 0; x < m; ++x)
            for (int b = 0; b < m; ++b) {
                double v;
                if (2 * x + 1 < m)
                    v = sc * std::sin(pi * (x + 1) * (b + 1) / n);
                else if (2 * x + 1 == m)
                    v = (b & 1) ? 0.0 : ((b >> 1) & 1 ? -sc : sc);
                else
                    v = (b & 1) ? -S[(m - 1 - x) * m + b] : S[(m - 1 - x) * m + b];
                S[x * m + b] = v;
            }
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) {
                const double ca = 2.0 * std::cos(pi * (a + 1) / n), cb = 2.0 * std::cos(pi * (b + 1) / n);
                W5[a * m + b] = 1.0 / (1.0 - 0.25 * (ca + cb));
                Wc[a * m + b] = 1.0 / (1.0 - 0.2 * (ca + cb) - 0.05 * (ca * cb));
            }
    }
    for (int k = 0; k < kDirectTable; ++k) t32[k] = (float)t64[k];
    cudaError_t e = cudaMemcpyToSymbol(g_direct64, t64, sizeof(t64));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_direct32, t32, sizeof(t32));
    if (e == cudaSuccess) g_direct_ready[dev].store(true);
    return e;
}

cudaError_t init_mg_kernel_attributes() {
    cudaError_t e = set_attrs_t<double>();
    if (e == cudaSuccess) e = set_cluster_attrs_t<double>();
    if (e == cudaSuccess) e = set_cluster_attrs_t<float>();
    int dev = -1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxClusterDevices) g_cluster_size[dev].store(query_cluster_size());
    if (e == cudaSuccess) e = init_direct_tables(dev);
    if (e == cudaSuccess) e = set_attrs_t<float>();
    if (e == cudaSuccess) e = set_batch_attrs_t<0>();
    if (e == cudaSuccess) e = set_batch_attrs_t<1>();
    return e;
}

#define LCX_MG_INSTANTIATE(T)                                                                                          \
    template cudaError_t launch_down<T>(cudaStream_t, int, int, const T *, int, const T *, T *, int, int, T *, int,   \
                                        int, T);                                                                      \
    template cudaError_t launch_up<T>(cudaStream_t, int, int, const T *, const T *, const T *, int, T *, int, int,     \
                                      int, T, double *, Correct64, FinishArgs);                                       \
    template cudaError_t launch_coarse<T>(cudaStream_t, int, const T *, int, const T *, T *, int, int, int, int, int,  \
                                          int, T, double *, FinishArgs);                                              \
    template cudaError_t launch_coarse_cluster<T>(cudaStream_t, int, const T *, int, T *, int, int, int, int, int,    \
                                                  int, T, int, int);
LCX_MG_INSTANTIATE(double)
LCX_MG_INSTANTIATE(float)

}  // namespace lcx
