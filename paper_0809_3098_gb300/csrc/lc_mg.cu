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
//            held in shared memory.
//
// A tile owns an aligned block of TX x TY interior nodes and recomputes a halo
// around it.  Invalid values enter a tile from its edge and spread one
// neighbour per colour phase; with the colour orders used here the residual
// after nu sweeps is exact at distances >= (4 nu + 1, 2 nu + 1) from the edge
// for the compact operator and 2 nu + 1 for the 5-point one, which sets the
// halo.  Tiles read psi from one buffer and write another (ping-pong), so no
// tile ever sees a neighbour's half-updated values.
#include "lc_internal.h"

namespace lcx {

namespace {

template <typename T, int OP>
__device__ __forceinline__ T gs_local(const T *sp, const T *sg, int c, int LP) {
    T n4 = (sp[c + 1] + sp[c - 1]) + (sp[c + LP] + sp[c - LP]);
    if (OP == 1) {
        T d4 = (sp[c + LP + 1] + sp[c + LP - 1]) + (sp[c - LP + 1] + sp[c - LP - 1]);
        return fma(T(0.2), n4, fma(T(0.05), d4, sg[c]));
    }
    return fma(T(0.25), n4, sg[c]);
}

// Halo (x, y) a tile needs for a valid residual after nu sweeps.
__host__ __device__ inline int halo_x(int op, int nu) { return op == 1 ? 4 * nu + 1 : 2 * nu + 1; }
__host__ __device__ inline int halo_y(int op, int nu) { return 2 * nu + 1; }

// One colour phase over the tile's updatable nodes: local [1, LX-2] x
// [1, LY-2] intersected with the domain interior.  Block is 2-D.
template <typename T, int OP>
__device__ void tile_phase(T *sp, const T *sg, int LP, int LX, int LY, int gx0, int gy0, int N, int colour,
                           T beta) {
    if (OP == 1) {
        int pi = colour & 1, pj = colour >> 1;
        int x0 = ((gx0 + 1) & 1) == pi ? 1 : 2;
        int y0 = ((gy0 + 1) & 1) == pj ? 1 : 2;
        int nx = LX - 2 >= x0 ? (LX - 2 - x0) / 2 + 1 : 0;
        int ny = LY - 2 >= y0 ? (LY - 2 - y0) / 2 + 1 : 0;
        for (int yy = threadIdx.y; yy < ny; yy += blockDim.y) {
            int y = y0 + 2 * yy, gj = gy0 + y;
            if (gj < 1 || gj >= N) continue;
            for (int xx = threadIdx.x; xx < nx; xx += blockDim.x) {
                int x = x0 + 2 * xx, gi = gx0 + x;
                if (gi < 1 || gi >= N) continue;
                int c = y * LP + x;
                T v = gs_local<T, OP>(sp, sg, c, LP);
                if (beta != T(1)) v = fma(beta, v - sp[c], sp[c]);
                sp[c] = v;
            }
        }
    } else {
        int nx = (LX - 2) / 2 + 1;
        for (int y = 1 + threadIdx.y; y <= LY - 2; y += blockDim.y) {
            int gj = gy0 + y;
            if (gj < 1 || gj >= N) continue;
            int x0 = ((gx0 + 1 + gj) & 1) == colour ? 1 : 2;
            for (int xx = threadIdx.x; xx < nx; xx += blockDim.x) {
                int x = x0 + 2 * xx, gi = gx0 + x;
                if (x > LX - 2 || gi < 1 || gi >= N) continue;
                int c = y * LP + x;
                T v = gs_local<T, OP>(sp, sg, c, LP);
                if (beta != T(1)) v = fma(beta, v - sp[c], sp[c]);
                sp[c] = v;
            }
        }
    }
}

template <typename T, int OP>
__device__ void tile_sweeps(T *sp, const T *sg, int LP, int LX, int LY, int gx0, int gy0, int N, int nu, T beta) {
    int ncol = OP == 1 ? 4 : 2;
    for (int s = 0; s < nu; ++s)
        for (int col = 0; col < ncol; ++col) {
            tile_phase<T, OP>(sp, sg, LP, LX, LY, gx0, gy0, N, col, beta);
            __syncthreads();
        }
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
__global__ void __launch_bounds__(512)
    k_down(const T *__restrict__ psi_in, int zero_init, const T *__restrict__ g, T *__restrict__ psi_out, int N,
           int P, T *__restrict__ gc, int Pc, int nu, T beta) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sp = reinterpret_cast<T *>(smem_raw);
    int RX = halo_x(OP, nu), RY = halo_y(OP, nu);
    int LX = TX + 2 * RX + 1, LY = TY + 2 * RY + 1, LP = LX;
    T *sg = sp + LY * LP;
    int ox0 = 1 + blockIdx.x * TX, oy0 = 1 + blockIdx.y * TY;
    int gx0 = ox0 - RX, gy0 = oy0 - RY;
    for (int y = threadIdx.y; y < LY; y += blockDim.y) {
        int gj = gy0 + y;
        for (int x = threadIdx.x; x < LX; x += blockDim.x) {
            int gi = gx0 + x;
            T p = T(0), q = T(0);
            if (gi >= 0 && gi <= N && gj >= 0 && gj <= N) {
                size_t c = (size_t)gj * P + gi;
                if (!zero_init) p = psi_in[c];
                q = g[c];
            }
            sp[y * LP + x] = p;
            sg[y * LP + x] = q;
        }
    }
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
            sg[c] = interior ? gs_local<T, OP>(sp, sg, c, LP) - sp[c] : T(0);
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

// Prolongation + correction + post-smoothing; on the fine level also the
// tile's sum of rho^2 over its owner nodes (partials != nullptr).  With
// cor.psi64 set (the mixed-precision fine level) the smoothed correction is
// not stored: it is added to the FP64 solution, psi64 += e, and the FP32
// shadow of the new psi64 is written.
template <typename T, int OP, int TX, int TY>
__global__ void __launch_bounds__(512)
    k_up(const T *__restrict__ psi_in, const T *__restrict__ g, const T *__restrict__ ec, int Pc,
         T *__restrict__ psi_out, int N, int P, int nu, T beta, double *__restrict__ partials, Correct64 cor) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    T *sp = reinterpret_cast<T *>(smem_raw);
    int RX = halo_x(OP, nu), RY = halo_y(OP, nu);
    int LX = TX + 2 * RX + 1, LY = TY + 2 * RY + 1, LP = LX;
    T *sg = sp + LY * LP;
    int ox0 = 1 + blockIdx.x * TX, oy0 = 1 + blockIdx.y * TY;
    int gx0 = ox0 - RX, gy0 = oy0 - RY;
    for (int y = threadIdx.y; y < LY; y += blockDim.y) {
        int gj = gy0 + y;
        for (int x = threadIdx.x; x < LX; x += blockDim.x) {
            int gi = gx0 + x;
            T p = T(0), q = T(0);
            if (gi >= 0 && gi <= N && gj >= 0 && gj <= N) {
                size_t c = (size_t)gj * P + gi;
                p = psi_in[c];
                q = g[c];
                if (gi >= 1 && gi < N && gj >= 1 && gj < N) {
                    int I = gi >> 1, J = gj >> 1;
                    size_t cc = (size_t)J * Pc + I;
                    T e;
                    if (!(gi & 1) && !(gj & 1))
                        e = ec[cc];
                    else if ((gi & 1) && !(gj & 1))
                        e = T(0.5) * (ec[cc] + ec[cc + 1]);
                    else if (!(gi & 1) && (gj & 1))
                        e = T(0.5) * (ec[cc] + ec[cc + Pc]);
                    else
                        e = T(0.25) * ((ec[cc] + ec[cc + 1]) + (ec[cc + Pc] + ec[cc + Pc + 1]));
                    p += e;
                }
            }
            sp[y * LP + x] = p;
            sg[y * LP + x] = q;
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
                double pnew = cor.psi64[c64] + (double)sp[c];
                cor.psi64[c64] = pnew;
                cor.psi32[(size_t)gj * cor.P32 + gi] = (float)pnew;
            } else {
                psi_out[(size_t)gj * P + gi] = sp[c];
            }
            if (partials) {
                double r = (double)(gs_local<T, OP>(sp, sg, c, LP) - sp[c]);
                acc += r * r;
            }
        }
    }
    if (partials) {
        acc = block_sum2d(acc, red);
        if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = acc;
    }
}

// ---------------------------------------------------------------------------
// A V-cycle over levels N0, N0/2, ..., down to 2 or 3 intervals, in one block
// with every level in shared memory (pitch N_k + 1).  g_in: right-hand side of
// the top level; psi_warm: its initial guess (nullptr = zero); psi_out: where
// the top level's result goes; partial: if set, the sum of rho^2 of the top
// level after the cycle.
template <typename T, int OP>
__device__ void cs_phase(T *sp, const T *sg, int n, int colour, T beta) {
    int LP = n + 1, m = n - 1;
    int tid = threadIdx.x, nt = blockDim.x;
    if (OP == 1) {
        int pi = colour & 1, pj = colour >> 1;
        int x0 = pi ? 1 : 2, y0 = pj ? 1 : 2;
        int nx = m >= x0 ? (m - x0) / 2 + 1 : 0, ny = m >= y0 ? (m - y0) / 2 + 1 : 0;
        for (int k = tid; k < nx * ny; k += nt) {
            int x = x0 + 2 * (k % nx), y = y0 + 2 * (k / nx);
            int c = y * LP + x;
            T v = gs_local<T, OP>(sp, sg, c, LP);
            if (beta != T(1)) v = fma(beta, v - sp[c], sp[c]);
            sp[c] = v;
        }
    } else {
        int nx = m / 2 + 1;
        for (int k = tid; k < nx * m; k += nt) {
            int y = 1 + k / nx;
            int x = (((1 + y) & 1) == colour ? 1 : 2) + 2 * (k % nx);
            if (x > m) continue;
            int c = y * LP + x;
            T v = gs_local<T, OP>(sp, sg, c, LP);
            if (beta != T(1)) v = fma(beta, v - sp[c], sp[c]);
            sp[c] = v;
        }
    }
}

template <typename T, int OP>
__device__ void cs_sweeps(T *sp, const T *sg, int n, int nu, T beta) {
    for (int s = 0; s < nu; ++s)
        for (int col = 0; col < (OP == 1 ? 4 : 2); ++col) {
            cs_phase<T, OP>(sp, sg, n, col, beta);
            __syncthreads();
        }
}

template <typename T, int OP>
__global__ void __launch_bounds__(1024)
    k_coarse(const T *__restrict__ g_in, int Pg, const T *__restrict__ psi_warm, T *__restrict__ psi_out, int Po,
             int N0, int nl, int nu1, int nu2, int nuc, T beta, double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    T *base = reinterpret_cast<T *>(smem_raw);
    T *sp[kMaxLevels], *sg[kMaxLevels];
    int off = 0;
    for (int k = 0; k < nl; ++k) {
        int n = N0 >> k, sz = (n + 1) * (n + 1);
        sp[k] = base + off;
        sg[k] = base + off + sz;
        off += 2 * sz;
    }
    T *sr = base + off;  // residual scratch, (N0+1)^2
    int tid = threadIdx.x, nt = blockDim.x;
    for (int k = tid; k < off; k += nt) base[k] = T(0);
    __syncthreads();
    int L0 = N0 + 1;
    for (int k = tid; k < L0 * L0; k += nt) {
        int x = k % L0, y = k / L0;
        if (x >= 1 && x < N0 && y >= 1 && y < N0) {
            sg[0][k] = g_in[(size_t)y * Pg + x];
            if (psi_warm) sp[0][k] = psi_warm[(size_t)y * Po + x];
        }
    }
    __syncthreads();
    for (int k = 0; k + 1 < nl; ++k) {
        int n = N0 >> k, LP = n + 1, nc = n / 2, LPc = nc + 1;
        cs_sweeps<T, OP>(sp[k], sg[k], n, nu1, beta);
        for (int q = tid; q < LP * LP; q += nt) {
            int x = q % LP, y = q / LP;
            sr[q] = (x >= 1 && x < n && y >= 1 && y < n) ? gs_local<T, OP>(sp[k], sg[k], q, LP) - sp[k][q] : T(0);
        }
        __syncthreads();
        for (int q = tid; q < LPc * LPc; q += nt) {
            int X = q % LPc, Y = q / LPc;
            if (X >= 1 && X < nc && Y >= 1 && Y < nc) {
                const T *r = sr + (2 * Y) * LP + 2 * X;
                T e4 = (r[1] + r[-1]) + (r[LP] + r[-LP]);
                T d4 = (r[LP + 1] + r[LP - 1]) + (r[-LP + 1] + r[-LP - 1]);
                sg[k + 1][q] = fma(T(0.5), e4, fma(T(0.25), d4, r[0]));
            }
            sp[k + 1][q] = T(0);
        }
        __syncthreads();
    }
    cs_sweeps<T, OP>(sp[nl - 1], sg[nl - 1], N0 >> (nl - 1), nuc, beta);
    for (int k = nl - 2; k >= 0; --k) {
        int n = N0 >> k, LP = n + 1, LPc = n / 2 + 1;
        const T *ec = sp[k + 1];
        for (int q = tid; q < LP * LP; q += nt) {
            int i = q % LP, j = q / LP;
            if (i >= 1 && i < n && j >= 1 && j < n) {
                int I = i >> 1, J = j >> 1, cc = J * LPc + I;
                T e;
                if (!(i & 1) && !(j & 1))
                    e = ec[cc];
                else if ((i & 1) && !(j & 1))
                    e = T(0.5) * (ec[cc] + ec[cc + 1]);
                else if (!(i & 1) && (j & 1))
                    e = T(0.5) * (ec[cc] + ec[cc + LPc]);
                else
                    e = T(0.25) * ((ec[cc] + ec[cc + 1]) + (ec[cc + LPc] + ec[cc + LPc + 1]));
                sp[k][q] += e;
            }
        }
        __syncthreads();
        cs_sweeps<T, OP>(sp[k], sg[k], n, nu2, beta);
    }
    double acc = 0.0;
    for (int k = tid; k < L0 * L0; k += nt) {
        int x = k % L0, y = k / L0;
        if (x >= 1 && x < N0 && y >= 1 && y < N0) {
            psi_out[(size_t)y * Po + x] = sp[0][k];
            if (partial) {
                double r = (double)(gs_local<T, OP>(sp[0], sg[0], k, L0) - sp[0][k]);
                acc += r * r;
            }
        }
    }
    if (partial) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        int lane = tid & 31, warp = tid >> 5;
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (warp == 0) {
            acc = lane < (nt + 31) / 32 ? red[lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
            if (lane == 0) partial[0] = acc;
        }
    }
}

constexpr int kTBX = 32, kTBY = 16;  // 512 threads per tile block

template <typename T, int TX, int TY>
size_t down_smem(int op, int nu) {
    int LX = TX + 2 * halo_x(op, nu) + 1, LY = TY + 2 * halo_y(op, nu) + 1;
    return 2 * (size_t)LX * LY * sizeof(T);
}

template <typename T, int OP, int TX, int TY>
cudaError_t down_t(cudaStream_t s, const T *psi_in, int zero_init, const T *g, T *psi_out, int N, int P, T *gc, int Pc,
                   int nu, T beta) {
    size_t sm = down_smem<T, TX, TY>(OP, nu);
    auto kern = k_down<T, OP, TX, TY>;
    dim3 grid((N - 1 + TX - 1) / TX, (N - 1 + TY - 1) / TY);
    kern<<<grid, dim3(kTBX, kTBY), sm, s>>>(psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
    return cudaGetLastError();
}

template <typename T, int OP, int TX, int TY>
cudaError_t up_t(cudaStream_t s, const T *psi_in, const T *g, const T *ec, int Pc, T *psi_out, int N, int P, int nu,
                 T beta, double *partials, Correct64 cor) {
    size_t sm = down_smem<T, TX, TY>(OP, nu);
    auto kern = k_up<T, OP, TX, TY>;
    dim3 grid((N - 1 + TX - 1) / TX, (N - 1 + TY - 1) / TY);
    kern<<<grid, dim3(kTBX, kTBY), sm, s>>>(psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor);
    return cudaGetLastError();
}

}  // namespace

// Tile shape per level: large tiles (fewer recomputed halo nodes) where the
// level has enough of them to fill the GPU, small ones otherwise.
bool use_big_tiles(int N) { return ((N - 1 + 127) / 128) * ((N - 1 + 63) / 64) >= 120; }

int tiles_of(int N) {
    return use_big_tiles(N) ? ((N - 1 + 127) / 128) * ((N - 1 + 63) / 64) : ((N - 1 + 31) / 32) * ((N - 1 + 31) / 32);
}

size_t tile_smem_bytes(int N, int op, int nu, int elem) {
    int TX = use_big_tiles(N) ? 128 : 32, TY = use_big_tiles(N) ? 64 : 32;
    int LX = TX + 2 * halo_x(op, nu) + 1, LY = TY + 2 * halo_y(op, nu) + 1;
    return 2 * (size_t)LX * LY * elem;
}

template <typename T>
cudaError_t launch_down(cudaStream_t s, int op, const T *psi_in, int zero_init, const T *g, T *psi_out, int N, int P,
                        T *gc, int Pc, int nu, T beta) {
    bool big = use_big_tiles(N);
    if (op == 1)
        return big ? down_t<T, 1, 128, 64>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta)
                   : down_t<T, 1, 32, 32>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
    return big ? down_t<T, 0, 128, 64>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta)
               : down_t<T, 0, 32, 32>(s, psi_in, zero_init, g, psi_out, N, P, gc, Pc, nu, beta);
}

template <typename T>
cudaError_t launch_up(cudaStream_t s, int op, const T *psi_in, const T *g, const T *ec, int Pc, T *psi_out, int N,
                      int P, int nu, T beta, double *partials, Correct64 cor) {
    bool big = use_big_tiles(N);
    if (op == 1)
        return big ? up_t<T, 1, 128, 64>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor)
                   : up_t<T, 1, 32, 32>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor);
    return big ? up_t<T, 0, 128, 64>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor)
               : up_t<T, 0, 32, 32>(s, psi_in, g, ec, Pc, psi_out, N, P, nu, beta, partials, cor);
}

size_t coarse_smem_bytes(int N0, int nl, int elem) {
    size_t n = 0;
    for (int k = 0; k < nl; ++k) n += 2 * (size_t)((N0 >> k) + 1) * ((N0 >> k) + 1);
    n += (size_t)(N0 + 1) * (N0 + 1);
    return n * elem;
}

template <typename T>
cudaError_t launch_coarse(cudaStream_t s, int op, const T *g_in, int Pg, const T *psi_warm, T *psi_out, int Po, int N0,
                          int nl, int nu1, int nu2, int nuc, T beta, double *partial) {
    size_t sm = coarse_smem_bytes(N0, nl, sizeof(T));
    auto kern = op == 1 ? k_coarse<T, 1> : k_coarse<T, 0>;
    int threads = sizeof(T) == 8 ? 512 : 1024;
    kern<<<1, threads, sm, s>>>(g_in, Pg, psi_warm, psi_out, Po, N0, nl, nu1, nu2, nuc, beta, partial);
    return cudaGetLastError();
}

// Raises every tile / coarse kernel's dynamic shared-memory limit once, before
// any launch or graph capture.
template <typename T>
static cudaError_t set_attrs_t() {
    const void *k[] = {(const void *)k_down<T, 0, 128, 64>, (const void *)k_down<T, 1, 128, 64>,
                       (const void *)k_down<T, 0, 32, 32>,  (const void *)k_down<T, 1, 32, 32>,
                       (const void *)k_up<T, 0, 128, 64>,   (const void *)k_up<T, 1, 128, 64>,
                       (const void *)k_up<T, 0, 32, 32>,    (const void *)k_up<T, 1, 32, 32>,
                       (const void *)k_coarse<T, 0>,        (const void *)k_coarse<T, 1>};
    for (const void *f : k) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxSmem - 1024));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t init_mg_kernel_attributes() {
    cudaError_t e = set_attrs_t<double>();
    return e == cudaSuccess ? set_attrs_t<float>() : e;
}

#define LCX_MG_INSTANTIATE(T)                                                                                          \
    template cudaError_t launch_down<T>(cudaStream_t, int, const T *, int, const T *, T *, int, int, T *, int, int, T); \
    template cudaError_t launch_up<T>(cudaStream_t, int, const T *, const T *, const T *, int, T *, int, int, int, T,   \
                                      double *, Correct64);                                                           \
    template cudaError_t launch_coarse<T>(cudaStream_t, int, const T *, int, const T *, T *, int, int, int, int, int,  \
                                          int, T, double *);
LCX_MG_INSTANTIATE(double)
LCX_MG_INSTANTIATE(float)

}  // namespace lcx
