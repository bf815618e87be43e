// Internal declarations shared by the library's CUDA translation units.
//
// Device data layout: every level-l field is (N_l+1) x (N_l+1) nodes stored
// row-major with a row pitch P_l (elements, a multiple of 32) so that each row
// starts on a 256-byte boundary; element (i, j) is at j*P_l + i, with i the x
// index and j the y index (j = N_l is the lid).
//
// The multigrid works in a scaled form.  With kappa = 3/10 for the compact
// operator and 1/4 for the 5-point operator, the stored right-hand side is
// g = -kappa h^2 f, the Gauss-Seidel value of node P is
//     compact:  0.2 * sum(edge neighbours) + 0.05 * sum(diagonal neighbours) + g_P
//     5-point:  0.25 * sum(edge neighbours) + g_P
// (the SOR update of Eq. (15) at beta = 1, divided through by its diagonal),
// the local residual is rho = (Gauss-Seidel value) - psi_P, so that
// f - L_h psi = -rho / (kappa h^2), and full-weighting the fine residual onto
// the coarse grid gives the coarse scaled right-hand side g_c = 4 R(rho).
// Relative residual norms are scale-free: ||rho|| / ||g|| = ||f - L psi|| / ||f||.
// Every kernel sums neighbours in the same order, (E + W) + (N + S) and
// (NE + SE) + (NW + SW) (column pairs, which a kernel can share between
// neighbouring columns), so all execution modes give the same bits and the
// scheme stays exactly equivariant under the mirror x -> 1 - x.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include <nvtx3/nvToolsExt.h>  // header-only NVTX: ranges for profilers, no-ops without one

namespace lcx {

// Profiler range for the enclosing scope (NVTX push / pop).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kLogN = 65536;
constexpr int kMaxLevels = 16;

constexpr int kStatusNoConv = 1;
constexpr int kStatusNonFinite = 2;
constexpr int kStatusTimeout = 4;  // a bounded device-side wait gave up

// Device-resident solver state, one per context.
struct DevState {
    int cycles;       // V-cycles done in the solve in progress
    int status;       // kStatus* bits, sticky until read by the host
    int last_cycles;  // cycles of the last finished solve
    int more;         // eager mode: 1 if the V-cycle loop goes on
    double last_rel;  // relative residual at the end of the last solve
    unsigned long long nsolves;
    double mon[3];    // max|d omega|/dt, RES_psi, RES_omega
    unsigned int arrive;  // blocks that have written their residual partial (fused finisher)
    unsigned int pad1;
    unsigned int bar_count, bar_gen;  // fused smoother's grid barrier: arrivals, and blocks that have left
    int log[kLogN];   // cycles per solve, ring buffer indexed by nsolves
};

// Coefficients of one SSPRK(5,4) stage in low-storage form.
//   mode 0: out = a0 W0 + a1 in + bdt L
//   mode 1: as mode 0, and acc = acc_in * in
//   mode 2: as mode 0, and acc = acc + acc_in * in + acc_L * L
//   mode 3: out = acc + a1 in + bdt L
struct StageCoef {
    double a0, a1, bdt, acc_in, acc_L;
    int mode;
};

// ---- programmatic dependent launch (PDL)
// Every kernel of the step starts with pdl_enter(): it waits until the
// previous kernel in the stream has finished and its writes are visible.
// Launched with the programmatic-stream-serialization attribute (launch_pdl
// under a PdlScope), a kernel is launched once its predecessor's blocks have
// all exited, without waiting for the predecessor's completion to be
// processed, and nothing touches global memory before the wait; for a kernel
// launched without the attribute the wait does nothing.  No kernel triggers
// its dependents early: an explicit trigger at kernel entry, which lets the
// next grid's blocks occupy the SMs while the current one runs, made the
// FP64 step 25% slower on GB300, where this form saves 1-2%.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

extern thread_local int tl_pdl;
struct PdlScope {
    int prev;
    explicit PdlScope(int on) : prev(tl_pdl) { tl_pdl = on; }
    ~PdlScope() { tl_pdl = prev; }
    PdlScope(const PdlScope &) = delete;
    PdlScope &operator=(const PdlScope &) = delete;
};

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = tl_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// Arguments of the end-of-cycle decision that the last block of a kernel
// producing residual partials takes (enabled = 0: partials only).  The last
// block sums the nr residual partials and the ng right-hand-side partials in
// a fixed order, applies the stopping rule ||rho|| <= tol ||g|| (after every
// cycle; NaN/Inf or max_cycles end the loop with a status bit) and either
// sets the graph while-node's condition (h != 0) or writes ds->more (eager).
struct FinishArgs {
    int enabled;
    int nr;
    const double *gpart;
    int ng;
    DevState *ds;
    cudaGraphConditionalHandle h;
    double tol;
    int max_cycles;
};

#ifdef __CUDACC__
// FP64 <-> FP32 conversions on the integer pipes.  On GB300 the hardware
// conversions run on the FP64 unit (~64 clocks per warp instruction, about 2
// lane conversions per clock per SM, the rate of a DADD), so in kernels
// bound by that unit they cost as much as the arithmetic.  These give the
// hardware's bits with integer instructions: f64_to_f32 rounds to nearest,
// ties to even, with the same overflow to infinity and the same subnormal
// results; f32_to_f64 is exact.  NaN in gives a NaN (payload not kept).
// lc_selftest_conversions compares both with the hardware conversions.
__device__ __forceinline__ float f64_to_f32(double d) {
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    if (e == 0x7ff) return __uint_as_float(sign | (((hi & 0xfffffu) | lo) ? 0x7fc00000u : 0x7f800000u));
    const int E = e - 896;  // exponent field of the float: 1023 - 127 = 896
    if (E >= 255) return __uint_as_float(sign | 0x7f800000u);
    if (E >= 1) {  // normal result: top 23 of the 52 mantissa bits, round on the other 29
        const unsigned m23 = ((hi & 0xfffffu) << 3) | (lo >> 29), rem = lo & 0x1fffffffu;
        const unsigned up = rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u));
        return __uint_as_float(sign | ((((unsigned)E << 23) | m23) + up));  // a carry moves into the exponent
    }
    // subnormal or zero result: the value is m53 2^(e - 1075), the result k 2^-149
    if (e == 0) return __uint_as_float(sign);  // an FP64 subnormal is far below 2^-150
    const int sh = 926 - e;                    // >= 30
    if (sh > 54) return __uint_as_float(sign);
    const unsigned long long m53 = (1ull << 52) | ((unsigned long long)(hi & 0xfffffu) << 32) | lo;
    const unsigned long long k = m53 >> sh, rem = m53 & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    const unsigned up = rem > half || (rem == half && (k & 1ull));
    return __uint_as_float(sign | (unsigned)(k + up));
}

__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    int e = (int)((u >> 23) & 0xffu);
    unsigned m = u & 0x7fffffu;
    if (e == 0xff) return __hiloint2double((int)(sign | 0x7ff00000u | (m ? 0x80000u : 0u)), 0);
    if (e == 0) {
        if (m == 0) return __hiloint2double((int)sign, 0);
        const int sh = __clz(m) - 8;  // moves the leading one to bit 23
        m = (m << sh) & 0x7fffffu;
        e = 1 - sh;
    }
    return __hiloint2double((int)(sign | ((unsigned)(e + 896) << 20) | (m >> 3)), (int)(m << 29));
}

template <typename T>
__device__ __forceinline__ double to_f64(T v);
template <>
__device__ __forceinline__ double to_f64<double>(double v) {
    return v;
}
template <>
__device__ __forceinline__ double to_f64<float>(float v) {
    return f32_to_f64(v);
}

// Rounded products and sums that the compiler may not fuse into an FMA: the
// prolongation's e = w (a + b) and psi += e are written with these in every
// kernel, so that all kernels round them alike.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Scaled residual rho = (Gauss-Seidel value) - psi of node (i, j),
// i = i0 - 1 + lane, for a warp over 32 consecutive columns of row j >= 1
// (blockDim.x = 32); lanes 0 and 31 are halo and only supply column data.
// Compact operator: with the column sums V(k) = psi(k, j+1) + psi(k, j-1) and
// H(k) = 4 psi(k, j) + V(k),
//   GS = 0.2 n4 + 0.05 d4 + g = 0.05 (H(i+1) + H(i-1) + 4 V(i)) + g,
// six FP64 operations per node instead of seven, mirror-image terms still
// paired; H(i +- 1) come from the neighbouring lanes.  5-point: 0.25 n4 + g
// with n4 = (E + W) + V(i).  Returns whether (i, j) is an interior node.
template <typename T, int OP>
__device__ __forceinline__ bool rho_halo(const T *__restrict__ psi, const T *__restrict__ g, int N, int P, int i0,
                                         int j, T &rho) {
    int lane = threadIdx.x & 31;
    int i = i0 - 1 + lane;
    bool rowok = j < N;
    size_t c = (size_t)j * P + i;
    T p = T(0), V = T(0);
    if (rowok && i <= N) {
        p = psi[c];
        V = psi[c + P] + psi[c - P];
    }
    bool act = rowok && lane >= 1 && lane <= 30 && i < N;
    if (OP == 1) {
        T H = fma(T(4), p, V);
        T Hr = __shfl_down_sync(0xffffffffu, H, 1), Hl = __shfl_up_sync(0xffffffffu, H, 1);
        if (!act) return false;
        rho = fma(T(0.05), fma(T(4), V, Hr + Hl), g[c] - p);
    } else {
        T E = __shfl_down_sync(0xffffffffu, p, 1), W = __shfl_up_sync(0xffffffffu, p, 1);
        if (!act) return false;
        rho = fma(T(0.25), (E + W) + V, g[c]) - p;
    }
    return true;
}

// rho = GS - psi at node c of an array with row pitch P, for the residuals
// that feed a restriction or a norm.  In FP64 the compact operator takes the
// H-form of rho_halo with the column sums formed at the node (same operands,
// order and rounding, so every FP64 residual of the library agrees bit for
// bit with rho_halo's); FP32, whose V-cycle kernels share the GS form, and
// the 5-point operator (where the two forms coincide) take GS - psi.
template <typename T, int OP, typename I>
__device__ __forceinline__ T rho_node(const T *p, const T *g, I c, int P) {
    if constexpr (OP == 1 && sizeof(T) == 8) {
        T V = p[c + P] + p[c - P];
        T Hr = fma(T(4), p[c + 1], p[c + 1 + P] + p[c + 1 - P]);
        T Hl = fma(T(4), p[c - 1], p[c - 1 + P] + p[c - 1 - P]);
        return fma(T(0.05), fma(T(4), V, Hr + Hl), g[c] - p[c]);
    } else {
        T n4 = (p[c + 1] + p[c - 1]) + (p[c + P] + p[c - P]);
        if (OP == 1) {
            T d4 = (p[c + P + 1] + p[c - P + 1]) + (p[c + P - 1] + p[c - P - 1]);
            return fma(T(0.2), n4, fma(T(0.05), d4, g[c])) - p[c];
        }
        return fma(T(0.25), n4, g[c]) - p[c];
    }
}

__device__ __forceinline__ double finish_block_sum(double v, double *sh) {
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
    return r;  // valid in thread 0
}

// Called by every thread of every block after thread 0 of the block has
// stored the block's residual partial; the last block of the grid to arrive
// takes the decision described at FinishArgs.
__device__ __forceinline__ void finish_if_last(const double *partials, FinishArgs fin) {
    __shared__ unsigned int s_last;
    __shared__ double s_red[32];
    int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    unsigned int nb = gridDim.x * gridDim.y;
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&fin.ds->arrive, 1u) == nb - 1 ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double sr = 0.0, sg = 0.0;
    for (int k = tid; k < (int)nb; k += nt) sr += __ldcg(partials + k);  // one partial per block
    for (int k = tid; k < fin.ng; k += nt) sg += __ldcg(fin.gpart + k);
    sr = finish_block_sum(sr, s_red);
    sg = finish_block_sum(sg, s_red);
    if (tid != 0) return;
    DevState *ds = fin.ds;
    ds->arrive = 0;
    int cyc = ds->cycles + 1;
    double rn = sqrt(sr), gn = sqrt(sg);
    bool finite = isfinite(rn) && isfinite(gn);
    unsigned int more = 0;
    if (!finite) {
        ds->status |= kStatusNonFinite;
    } else if (rn <= fin.tol * gn) {
    } else if (cyc >= fin.max_cycles) {
        ds->status |= kStatusNoConv;
    } else {
        more = 1;
    }
    if (more) {
        ds->cycles = cyc;
    } else {
        ds->cycles = 0;
        ds->last_cycles = cyc;
        ds->last_rel = gn > 0.0 ? rn / gn : (rn > 0.0 ? INFINITY : 0.0);
        ds->log[ds->nsolves % kLogN] = cyc;
        ds->nsolves += 1;
    }
    if (fin.h)
        cudaGraphSetConditional(fin.h, more);
    else
        ds->more = (int)more;
}
#endif

// ---- launchers (lc_kernels.cu); each enqueues on `s` and returns the launch error
template <typename T>
cudaError_t launch_smooth_colour(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int colour, T beta);
template <typename T>
cudaError_t launch_residual_restrict(cudaStream_t s, int op, const T *psi, const T *g, int Nf, int Pf, T *gc,
                                     T *psic, int Pc);
template <typename T>
cudaError_t launch_prolong_correct(cudaStream_t s, T *psi, int Nf, int Pf, const T *ec, int Pc);
template <typename T>
cudaError_t launch_coarsest(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int nsweeps, T beta);
template <typename T>
cudaError_t launch_residual_norm(cudaStream_t s, int op, const T *psi, const T *g, int N, int P, double *partials,
                                 FinishArgs fin);

// Residual kernels: a warp covers 32 consecutive columns of one row, the
// outer two lanes as halo, so a block of 32 x 8 threads owns kRX = 30 x 8
// interior nodes.
constexpr int kRX = 30, kRY = 8;
inline int residual_blocks_x(int N) { return (N - 1 + kRX - 1) / kRX; }
int residual_norm_blocks(int N);
// k_residual_norm (the FP64 stopping test) sums kNormRows rows per thread;
// its launch has residual_norm64_blocks(N) <= residual_norm_blocks(N) blocks.
constexpr int kNormRows = 4;
int residual_norm64_blocks(int N);
// nsweeps colour sweeps of the fine-level smoother in one cooperative launch
// of `blocks` co-resident blocks of 256 threads, a bounded grid barrier
// between colour phases (same values as launch_smooth_colour, bit for bit).
// extra: additional arrivals the barrier waits for (0; 1 only in the test
// that makes the wait run out).
template <typename T>
cudaError_t launch_smooth_fused(cudaStream_t s, int op, T *psi, const T *g, int N, int P, int nsweeps, T beta,
                                DevState *ds, int blocks, int extra);
// Co-resident blocks of the fused smoother on the current device (0 if the
// device cannot launch cooperative kernels).
int smooth_fused_blocks(int op, bool relax);
// Blocks of the fused smoother for a level of N intervals: one warp-sized
// item per warp, at most nmax (the co-resident limit).
int smooth_fused_level_blocks(int op, int N, int nmax);
// nsw lexicographic SOR sweeps (Eq. (15) in its superscripts' order) in one
// block, pipelined over wavefronts; psi in shared memory when
// sor_smem_bytes(N, P) <= kMaxSmem.
cudaError_t launch_sor_lex(cudaStream_t s, int op, double *psi, const double *g, int N, int P, int nsw, double beta);
size_t sor_smem_bytes(int N, int P);
cudaError_t init_sor_kernel_attributes();
// k_assemble_rhs keeps one row per thread: its partial sums of g^2 then
// follow the 32 x 8 tiles of the batched assembly, so single and batched
// cavities compare their residuals with the same ||g||.
int assemble_blocks(int N);
int monitor_blocks(int N);

cudaError_t launch_assemble_rhs(cudaStream_t s, int op, const double *omega, double *g, int N, int P, double *gpart);
cudaError_t launch_thom(cudaStream_t s, const double *psi, double *W0, double *Wa, double *Wb, int N, int P, double U,
                        int profile);
cudaError_t launch_rhs_stage(cudaStream_t s, const double *psi, const double *in, const double *W0, double *acc,
                             double *out, int N, int P, double Re, int advect, StageCoef c);
cudaError_t launch_monitor(cudaStream_t s, const double *psi0, const double *psi1, const double *w0, const double *w1,
                           int N, int P, double *part, DevState *ds, double dt);
cudaError_t launch_zero_walls(cudaStream_t s, double *psi, int N, int P);

// FP64 correction target of the mixed-precision fine level (psi64 == nullptr:
// none; psi32 == nullptr: the FP32 shadow is refreshed after the solve).
struct Correct64 {
    double *psi64;
    int P64;
    float *psi32;
    int P32;
};

// ---- shared-memory multigrid kernels (lc_mg.cu)
// Tile shapes (owned nodes): shared-memory tiles 0 = 110x54, 1 = 110x22,
// 2 = 46x22, 3 = 16x16; 4 = 44x20 register tiles, one per warp (lc_warp.cu;
// FP32 only, nu <= 2 for the compact operator, so tile_smem_bytes reports it
// as not fitting otherwise).  tile_shape_for picks one per level (force >= 0
// overrides when the shape fits).
int tile_shape_for(int N, int op, int nu, int elem, int force);
int tile_tx(int shape);
int tile_ty(int shape);
int tiles_of(int N, int shape);
size_t tile_smem_bytes(int shape, int op, int nu, int elem);
size_t coarse_smem_bytes(int N0, int nl, int elem);
template <typename T>
cudaError_t launch_down(cudaStream_t s, int shape, int op, const T *psi_in, int zero_init, const T *g, T *psi_out,
                        int N, int P, T *gc, int Pc, int nu, T beta);
template <typename T>
cudaError_t launch_up(cudaStream_t s, int shape, int op, const T *psi_in, const T *g, const T *ec, int Pc, T *psi_out,
                      int N, int P, int nu, T beta, double *partials, Correct64 cor, FinishArgs fin);
template <typename T>
cudaError_t launch_coarse(cudaStream_t s, int op, const T *g_in, int Pg, const T *psi_warm, T *psi_out, int Po, int N0,
                          int nl, int nu1, int nu2, int nuc, T beta, double *partial, FinishArgs fin);

// The coarse V-cycle on a cluster of C blocks (lc_mg.cu): levels of more
// than `split` intervals split by rows over the blocks, the rest in block 0;
// the same values as launch_coarse with psi_warm = nullptr and no norm.
size_t cluster_smem_bytes(int N0, int nl, int C, int split, int elem);
template <typename T>
cudaError_t launch_coarse_cluster(cudaStream_t s, int op, const T *g_in, int Pg, T *psi_out, int Po, int N0, int nl,
                                  int nu1, int nu2, int nuc, T beta, int C, int split);
int coarse_cluster_size(int device);  // 16, 8, or 0 (device cannot run it, or before init_mg_kernel_attributes on it)

constexpr size_t kMaxSmem = 227 * 1024;
cudaError_t init_mg_kernel_attributes();

// ---- register-tile (warp tile) FP32 multigrid kernels (lc_warp.cu)
bool warp_tile_fits(int op, int nu);
int warp_tile_blocks(int N);  // blocks of 4 warp tiles for one level of N intervals
cudaError_t launch_down_warp(cudaStream_t s, int op, const float *g, float *e_out, int N, int P, float *gc, int Pc,
                             int nu, float beta);
cudaError_t launch_up_warp(cudaStream_t s, int op, const float *e_in, const float *g, const float *ec, int Pc,
                           float *e_out, int N, int P, int nu, float beta, Correct64 cor);


// ---- mixed-precision kernels (lc_mixed.cu)
cudaError_t launch_residual64_to32(cudaStream_t s, int op, const double *psi64, const double *g64, int N, int P64,
                                   float *r32, int P32, double *partials, FinishArgs fin);
cudaError_t launch_correct64(cudaStream_t s, const float *e32, int Pe, double *psi64, int P64, float *psi32, int P32,
                             int N);
cudaError_t launch_rhs_stage_mixed(cudaStream_t s, const float *psi32, int Ps, const float *in32, const double *in64,
                                   const double *W0, double *acc, double *out64, float *out32, int N, int P64, int P32,
                                   double Re, int advect, StageCoef c);
cudaError_t launch_thom_mixed(cudaStream_t s, const double *psi64, double *const w64[3], float *const w32[3], int N,
                              int P64, int P32, double U, int profile);
cudaError_t launch_to32(cudaStream_t s, const double *src, int P64, float *dst, int P32, int N);
// Compares f64_to_f32 / f32_to_f64 with the hardware conversions on n test
// values; bad[0], bad[1] count the mismatches of each direction.
cudaError_t launch_selftest_conversions(cudaStream_t s, long long n, unsigned long long seed,
                                        unsigned long long *bad);

// ---- batched engine (lc_batch.cu host side; kernels in lc_mg.cu and lc_mixed.cu)
constexpr int kMaxBatch = 256;

// One cavity of a batch (device memory; the solve state fields change on the
// device).  Mixed precision: the fine level holds psi64/g64 (FP64) and the
// FP32 correction hierarchy eA/eB/g32 (g32[0] is the FP32 residual).
struct BatchCav {
    int N, nlev, lc;  // intervals, levels the V-cycle visits, first level of the one-block coarse cycle
    int P[kMaxLevels];
    double Re, dt;
    double *psi64, *g64;
    float *psi32;
    float *eA[kMaxLevels], *eB[kMaxLevels], *g32[kMaxLevels];
    double *W[4];  // W0, Wa, Wb, ACC
    float *Ws[3];  // FP32 shadows of W0, Wa, Wb
    int *log;      // cycles per solve, ring of kLogN
    // per-cavity constants, computed on the host as the single-cavity
    // launchers compute them (no division in the kernels)
    double h2, nu_invh2;  // h^2 and N^2 / Re
    float nu_invh2f;      // (float)(N^2 / Re)
    int pad0;
    // solve state
    int active, cycles, status, last_cycles;
    unsigned int arrive;
    int pad;
    double last_rel;
    unsigned long long nsolves;
};

// Block ranges of one batched launch: cavity c owns blocks [start[c], start[c+1])
// laid out as gx[c] blocks per row.
struct BatchRange {
    int count;
    int start[kMaxBatch + 1];
    int gx[kMaxBatch];
};

// Batch-wide loop state.
struct BatchState {
    unsigned int cav_arrive;  // cavities whose decision is taken this cycle
    int more;                 // eager mode: 1 if any cavity's loop goes on
    int any_status;
    int pad;
};

#ifdef __CUDACC__
// Cavity and block coordinates of this block in a batched launch.
__device__ __forceinline__ int batch_locate(const BatchRange *r, int &bx, int &by) {
    int b = blockIdx.x, lo = 0, hi = r->count;  // start[lo] <= b < start[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (r->start[mid] <= b) lo = mid;
        else hi = mid;
    }
    int local = b - r->start[lo];
    bx = local % r->gx[lo];
    by = local / r->gx[lo];
    return lo;
}
#endif

struct BatchFinish {
    int enabled;
    double tol;
    int max_cycles;
    cudaGraphConditionalHandle h;
    BatchState *bs;
};

// batched kernels
template <typename T>
cudaError_t launch_down_batch(cudaStream_t s, int shape, int op, BatchCav *cav, const BatchRange *r, int level,
                              int nblocks, int nu, T beta);
template <typename T>
cudaError_t launch_up_batch(cudaStream_t s, int shape, int op, BatchCav *cav, const BatchRange *r, int level,
                            int nblocks, int nu, T beta);
cudaError_t launch_coarse_batch(cudaStream_t s, int op, BatchCav *cav, int count, int smem, int nu1, int nu2, int nuc,
                                float beta);
cudaError_t launch_down_warp_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, int level, int nblocks,
                                   int nu, float beta);
cudaError_t launch_up_warp_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, int level, int nblocks,
                                 int nu, float beta);
cudaError_t launch_stage_batch(cudaStream_t s, BatchCav *cav, const BatchRange *r, int nblocks, int stage,
                               int advect, int rhs64);
cudaError_t launch_assemble_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, int nblocks, int stage,
                                  double *gpart);
// r: the residual range (blocks of kRX x kRY nodes); rg: the stage range, whose
// blocks wrote gpart.
cudaError_t launch_residual_batch(cudaStream_t s, int op, BatchCav *cav, const BatchRange *r, const BatchRange *rg,
                                  int nblocks, double *rpart, const double *gpart, BatchFinish fin);
cudaError_t launch_thom_batch(cudaStream_t s, BatchCav *cav, int count, double U);
cudaError_t launch_psi32_batch(cudaStream_t s, BatchCav *cav, const BatchRange *r, int nblocks);

// Sets the calling thread's lc_last_error() message.
void set_last_error(const char *msg);

}  // namespace lcx
