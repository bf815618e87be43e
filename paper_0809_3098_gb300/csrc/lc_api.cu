// C ABI of the cavity library (declared in include/lc.h): context, device
// workspace, the per-step CUDA graph and the host entry points.
//
// One time step is captured once into a CUDA graph and replayed:
//   for stage k = 1..5 (Eqs. (9)-(13)):
//     fused L(omega) + stage combination            (k_rhs_stage)
//     Poisson right-hand side from the new omega    (k_assemble_rhs, Eq. (14)/(17))
//     while-node: V-cycle; residual norm; finisher  (Eq. (15) smoother, stopping rule)
//     Thom wall vorticity                           (k_thom, Eq. (25))
// The V-cycle loop is a CUDA graph conditional while-node whose condition is
// set on the device by the finisher, so a solve never returns to the host.
#include "lc_internal.h"

#include "../../include/lc.h"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

using namespace lcx;

namespace {

thread_local std::string g_err;
std::mutex g_live_mu;
std::set<const void *> g_live;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return LC_ERR_CUDA;
}

#define LC_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// SSPRK(5,4) Shu-Osher coefficients, Eqs. (9)-(13).  The omega^(1) weight of
// Eq. (10) is printed 0.555626506348765; the stage's weights sum to one, so it
// is 1 - 0.444370493651235 = 0.555629506348765.  Eq. (9)'s 11-digit
// 0.39175222657 is carried to 0.391752226571890.
constexpr double A20 = 0.444370493651235, A21 = 0.555629506348765;
constexpr double A30 = 0.620101851488403, A32 = 0.379898148511597;
constexpr double A40 = 0.178079954393132, A43 = 0.821920045606868;
constexpr double A52 = 0.517231671970585, A53 = 0.096059710526147, A54 = 0.386708617503269;
constexpr double B10 = 0.391752226571890, B21 = 0.368410593050371, B32 = 0.251891774271694;
constexpr double B43 = 0.544974750228521, B53 = 0.063692468666290, B54 = 0.226007483236906;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
int pitch_of(int N) { return ((N + 1 + 31) / 32) * 32; }

int level_count(int N) {
    int n = 1;
    while (N % 2 == 0 && N >= 4) {
        N /= 2;
        ++n;
    }
    return (N == 2 || N == 3 || N == 5 || N == 7) ? n : -1;
}

bool valid_N(int N) { return N >= 8 && N <= 8192 && level_count(N) >= 2; }

// Offsets of every device array inside one workspace block.  FP64 arrays of
// level l have N_l + 1 rows of pitch Pl[l] elements; FP32 arrays use the same
// pitch in elements.
struct Layout {
    int nlev = 0, precision = 0;
    int Nl[kMaxLevels], Pl[kMaxLevels];
    size_t psi[kMaxLevels], psiB[kMaxLevels], g[kMaxLevels];  // FP64 (mixed: level 0 only)
    size_t eA[kMaxLevels], eB[kMaxLevels], g32[kMaxLevels];   // FP32 correction hierarchy (mixed)
    size_t psi32, r32;                                         // FP32 shadow of psi, FP32 residual (mixed)
    size_t W0, Wa, Wb, ACC, snap_psi, snap_w;
    size_t W0s, Was, Wbs;                                      // FP32 shadows of W0, Wa, Wb (mixed)
    size_t rpart, gpart, mpart, ds;
    int nrpart, nrpart_grid, ngpart, nmpart;
    size_t total = 0;
};

bool make_layout(int N, int precision, Layout &L) {
    if (!valid_N(N) || (precision != LC_PREC_FP64 && precision != LC_PREC_MIXED)) return false;
    L = Layout();
    L.nlev = level_count(N);
    L.precision = precision;
    bool mixed = precision == LC_PREC_MIXED;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    for (int l = 0; l < L.nlev; ++l) {
        L.Nl[l] = N >> l;
        L.Pl[l] = pitch_of(L.Nl[l]);
        size_t n = (size_t)(L.Nl[l] + 1) * L.Pl[l];
        if (!mixed || l == 0) {
            L.psi[l] = take(n * sizeof(double));
            L.g[l] = take(n * sizeof(double));
        }
        if (!mixed) L.psiB[l] = take(n * sizeof(double));
        if (mixed) {
            L.eA[l] = take(n * sizeof(float));
            L.eB[l] = take(n * sizeof(float));
            if (l > 0) L.g32[l] = take(n * sizeof(float));
        }
    }
    size_t n0 = (size_t)(N + 1) * L.Pl[0];
    if (mixed) {
        L.psi32 = take(n0 * sizeof(float));
        L.r32 = take(n0 * sizeof(float));
        L.W0s = take(n0 * sizeof(float));
        L.Was = take(n0 * sizeof(float));
        L.Wbs = take(n0 * sizeof(float));
    }
    L.W0 = take(n0 * sizeof(double));
    L.Wa = take(n0 * sizeof(double));
    L.Wb = take(n0 * sizeof(double));
    L.ACC = take(n0 * sizeof(double));
    L.snap_psi = take(n0 * sizeof(double));
    L.snap_w = take(n0 * sizeof(double));
    L.nrpart_grid = residual_norm_blocks(N);
    L.nrpart = L.nrpart_grid > tiles_of(N, 3) ? L.nrpart_grid : tiles_of(N, 3);  // the smallest tiles: the most partials
    L.ngpart = assemble_blocks(N);
    L.nmpart = monitor_blocks(N);
    L.rpart = take(L.nrpart * sizeof(double));
    L.gpart = take(L.ngpart * sizeof(double));
    L.mpart = take(3 * L.nmpart * sizeof(double) + 16);
    L.ds = take(sizeof(DevState));
    L.total = off;
    return true;
}

}  // namespace

void lcx::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

struct lc_ctx {
    int N;
    double Re, dt, tol;
    int op = LC_OP_COMPACT, precision = LC_PREC_FP64;
    int nu1 = 2, nu2 = 1, nuc = 16, max_cycles = 100, advect = 1, profile = 0, monitor = 0;
    int use_graph = 1;
    double beta = 1.1, U = 1.0;  // beta: the SOR relaxation of Eq. (15) in the smoother
    int solver = 0, sor_sweeps = 16;                    // 0 multigrid, 1 lexicographic SOR
    int coarse_direct = 1;  // the V-cycle ends at the first level below the fine one with <= 16 intervals, solved exactly
    int rhs64 = 1;  // mixed precision: L(omega) in FP64 (0: from the FP32 shadows)
    int fused = 0;                 // 1: fine-level FP64 colour phases of a pass in one cooperative launch
    int barrier_extra = 0;         // test hook: the fused kernel's barrier waits for this many more blocks
    int fused_blocks[2] = {0, 0};  // its grid (beta == 1, beta != 1); 0: not available
    int blocked = 1, coarse_max = -1;  // -1: 32 (FP64) or 64 (mixed)
    int fine_phases = kMaxLevels;     // FP64: levels above the coarse one with one launch per colour phase
    int tile_force = -1;                                // >= 0: one tile shape on every level
    int coarse_cluster = -1;  // coarse V-cycle on a cluster of this many blocks; -1: auto (FP64), 0: off
    int cluster_max = -1;     // first level run by the cluster kernel: N_l <= cluster_max (-1: 128)
    int cluster_split = 16;   // levels of <= cluster_split intervals run in the cluster's first block alone
    int pdl = 1;                   // launch the step's kernels with programmatic dependent launch
    bool pdl_unsupported = false;  // a graph with PDL edges failed to build: kernels launch one after another

    Layout lay;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false, initialized = false;
    int device = -1;

    cudaStream_t own_stream = nullptr, user_stream = nullptr;
    bool use_user_stream = false;
    cudaStream_t cap2 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_dirty = true;

    long long steps = 0;
    bool mon_valid = false;
    int kernels_per_cycle = 0, kernels_per_step = 0;

    cudaStream_t stream() const { return use_user_stream ? user_stream : own_stream; }
    template <typename T>
    T *at(size_t off) const {
        return reinterpret_cast<T *>(ws + off);
    }
    double *psi(int l) const { return at<double>(lay.psi[l]); }
    double *g(int l) const { return at<double>(lay.g[l]); }
    double *psiB(int l) const { return at<double>(lay.psiB[l]); }
    float *eA(int l) const { return at<float>(lay.eA[l]); }
    float *eB(int l) const { return at<float>(lay.eB[l]); }
    float *g32(int l) const { return l == 0 ? at<float>(lay.r32) : at<float>(lay.g32[l]); }
    bool mixed() const { return precision == LC_PREC_MIXED; }
    DevState *ds() const { return at<DevState>(lay.ds); }
};

namespace {

bool live(const lc_ctx *c) {
    std::lock_guard<std::mutex> lk(g_live_mu);
    return c && g_live.count(c);
}

#define LC_CHECK_CTX(c)                                           \
    do {                                                          \
        if (!live(c)) return fail(LC_ERR_ARG, "invalid context"); \
    } while (0)

void release_graph(lc_ctx *c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    c->graph_dirty = true;
}

// The level the V-cycle solves exactly: the first level below the fine one
// with at most 16 intervals (option coarse_direct), or -1 when the V-cycle
// goes down to the coarsest level (2, 3, 5 or 7 intervals) and smooths it.
constexpr int kDirectMaxN = 16;
int direct_level(const lc_ctx *c) {
    if (!c->coarse_direct) return -1;
    for (int l = 1; l < c->lay.nlev; ++l)
        if (c->lay.Nl[l] <= kDirectMaxN) return l;
    return -1;
}

// Levels the V-cycle visits, and the sweeps of its last level (0: the exact
// solve of the multigrid kernels' direct_level).
int vlevels(const lc_ctx *c) {
    int ld = direct_level(c);
    return ld >= 0 ? ld + 1 : c->lay.nlev;
}
int last_sweeps(const lc_ctx *c) { return direct_level(c) >= 0 ? 0 : c->nuc; }

// Blocks of the coarse cluster kernel; by default it runs in FP64 only (the
// FP32 one-block V-cycle is faster than the cluster's barriers).
int cluster_size(const lc_ctx *c) {
    if (c->coarse_cluster >= 0) return c->coarse_cluster;
    return c->mixed() ? 0 : coarse_cluster_size(c->device);
}

// Whether coarse level lc runs on the cluster kernel: it is not the fine level
// (whose last kernel takes the residual norm) and it has levels to split.
bool cluster_coarse(const lc_ctx *c, int lc) {
    int C = cluster_size(c), elem = c->mixed() ? 4 : 8;
    int cmax = c->cluster_max > 0 ? c->cluster_max : 128;
    const Layout &L = c->lay;
    return C > 0 && lc >= 1 && lc + 1 < vlevels(c) && L.Nl[lc] <= cmax && L.Nl[lc] > c->cluster_split &&
           cluster_smem_bytes(L.Nl[lc], vlevels(c) - lc, C, c->cluster_split, elem) <= kMaxSmem - 1024;
}

// First level handled by the coarse V-cycle kernel: the first level below the
// fine one that the cluster kernel takes (N_l <= cluster_max) when it is on,
// else the first with N_l <= coarse_max small enough for one block's shared
// memory.
int coarse_level(const lc_ctx *c) {
    const Layout &L = c->lay;
    const int nv = vlevels(c);
    int elem = c->mixed() ? 4 : 8;
    for (int l = 1; l < nv; ++l)
        if (cluster_coarse(c, l)) return l;
    int cmax = c->coarse_max > 0 ? c->coarse_max : (c->mixed() ? 64 : 32);
    for (int l = 0; l < nv; ++l)
        if (L.Nl[l] <= cmax && coarse_smem_bytes(L.Nl[l], nv - l, elem) <= kMaxSmem - 1024) return l;
    return nv - 1;
}

int tile_shape(const lc_ctx *c, int l) {
    int nu = c->nu1 > c->nu2 ? c->nu1 : c->nu2;
    return tile_shape_for(c->lay.Nl[l], c->op, nu, c->mixed() ? 4 : 8, c->tile_force);
}

// Whether the shared-memory tile kernels can run every level above the
// coarse level with the current smoothing counts.
bool blocked_ok(const lc_ctx *c) {
    if (!c->blocked && !c->mixed()) return false;
    int lc = coarse_level(c);
    int nu = c->nu1 > c->nu2 ? c->nu1 : c->nu2;
    for (int l = 0; l < lc; ++l)
        if (tile_smem_bytes(tile_shape(c, l), c->op, nu, c->mixed() ? 4 : 8) > kMaxSmem - 1024) return false;
    return true;
}

const FinishArgs kNoFinish{0, 0, nullptr, 0, nullptr, 0, 0.0, 0};

// One V-cycle with one launch per colour phase on every level (the plain
// form; used when blocked = 0 or the tiles would not fit in shared memory).
int enqueue_vcycle_phases(lc_ctx *c, cudaStream_t s) {
    const Layout &L = c->lay;
    const int nv = vlevels(c);
    int nc = c->op == LC_OP_COMPACT ? 4 : 2;
    c->kernels_per_cycle = (nv - 1) * ((c->nu1 + c->nu2) * nc + 2) + 1;
    for (int l = 0; l + 1 < nv; ++l) {
        for (int sw = 0; sw < c->nu1; ++sw)
            for (int col = 0; col < nc; ++col)
                LC_CUDA(launch_smooth_colour<double>(s, c->op, c->psi(l), c->g(l), L.Nl[l], L.Pl[l], col, c->beta));
        LC_CUDA(launch_residual_restrict<double>(s, c->op, c->psi(l), c->g(l), L.Nl[l], L.Pl[l], c->g(l + 1),
                                                 c->psi(l + 1), L.Pl[l + 1]));
    }
    int lc = nv - 1;
    if (direct_level(c) >= 0)  // the exact solve of the last level, as in the coarse kernels
        LC_CUDA(launch_coarse<double>(s, c->op, c->g(lc), L.Pl[lc], nullptr, c->psi(lc), L.Pl[lc], L.Nl[lc], 1,
                                      c->nu1, c->nu2, 0, c->beta, nullptr, kNoFinish));
    else
        LC_CUDA(launch_coarsest<double>(s, c->op, c->psi(lc), c->g(lc), L.Nl[lc], L.Pl[lc], c->nuc, c->beta));
    for (int l = nv - 2; l >= 0; --l) {
        LC_CUDA(launch_prolong_correct<double>(s, c->psi(l), L.Nl[l], L.Pl[l], c->psi(l + 1), L.Pl[l + 1]));
        for (int sw = 0; sw < c->nu2; ++sw)
            for (int col = 0; col < nc; ++col)
                LC_CUDA(launch_smooth_colour<double>(s, c->op, c->psi(l), c->g(l), L.Nl[l], L.Pl[l], col, c->beta));
    }
    return LC_OK;
}

// nsw smoothing sweeps of the fine FP64 level: one cooperative launch (the
// colour phases separated by a grid barrier) when available, else one launch
// per colour phase; the values are the same.  Returns the launch count, or a
// negative error code.
int enqueue_fine_sweeps(lc_ctx *c, cudaStream_t s, int nsw) {
    const Layout &L = c->lay;
    int nb = (c->fused & 1) ? c->fused_blocks[c->beta != 1.0 ? 1 : 0] : 0;
    if (nb > 0) {
        cudaError_t e = launch_smooth_fused<double>(s, c->op, c->psi(0), c->g(0), L.Nl[0], L.Pl[0], nsw, c->beta,
                                                    c->ds(), nb, c->barrier_extra);
        if (e != cudaSuccess) return cuda_fail(e, "launch_smooth_fused");
        return 1;
    }
    int nc = c->op == LC_OP_COMPACT ? 4 : 2, k = 0;
    for (int sw = 0; sw < nsw; ++sw)
        for (int col = 0; col < nc; ++col, ++k) {
            cudaError_t e = launch_smooth_colour<double>(s, c->op, c->psi(0), c->g(0), L.Nl[0], L.Pl[0], col, c->beta);
            if (e != cudaSuccess) return cuda_fail(e, "launch_smooth_colour");
        }
    return k;
}

// nsw smoothing sweeps of level l with one launch per colour phase (the fine
// level may take the fused form); returns the launch count or an error code.
int level_sweeps(lc_ctx *c, cudaStream_t s, int l, int nsw) {
    if (l == 0) return enqueue_fine_sweeps(c, s, nsw);
    const Layout &L = c->lay;
    int nmax = (c->fused & 2) ? c->fused_blocks[c->beta != 1.0 ? 1 : 0] : 0;
    if (nmax > 0) {  // one cooperative launch, as few blocks as the level's rows need
        cudaError_t e = launch_smooth_fused<double>(s, c->op, c->psi(l), c->g(l), L.Nl[l], L.Pl[l], nsw, c->beta,
                                                    c->ds(), smooth_fused_level_blocks(c->op, L.Nl[l], nmax),
                                                    c->barrier_extra);
        if (e != cudaSuccess) return cuda_fail(e, "launch_smooth_fused");
        return 1;
    }
    int nc = c->op == LC_OP_COMPACT ? 4 : 2, k = 0;
    for (int sw = 0; sw < nsw; ++sw)
        for (int col = 0; col < nc; ++col, ++k) {
            cudaError_t e = launch_smooth_colour<double>(s, c->op, c->psi(l), c->g(l), L.Nl[l], L.Pl[l], col, c->beta);
            if (e != cudaSuccess) return cuda_fail(e, "launch_smooth_colour");
        }
    return k;
}

FinishArgs finish_args(const lc_ctx *c, int nr, cudaGraphConditionalHandle h) {
    const Layout &L = c->lay;
    return FinishArgs{1, nr, c->at<double>(L.gpart), L.ngpart, c->ds(), h, c->tol, c->max_cycles};
}

// Enqueues one FP64 V-cycle on stream s.  When the cycle's last kernel writes
// the fine-level residual partials it also takes the end-of-cycle decision
// (*norm_done = true); otherwise the caller adds the residual-norm kernel.
int enqueue_vcycle(lc_ctx *c, cudaStream_t s, bool *norm_done, cudaGraphConditionalHandle h) {
    *norm_done = false;
    if (!blocked_ok(c)) return enqueue_vcycle_phases(c, s);
    const Layout &L = c->lay;
    int lc = coarse_level(c);
    const int nph = c->fine_phases < lc ? c->fine_phases : lc;  // finest levels with one launch per phase
    double *rpart = c->at<double>(L.rpart);
    int k = 0;
    for (int l = 0; l < lc; ++l) {
        if (l < nph) {
            int n = level_sweeps(c, s, l, c->nu1);
            if (n < 0) return n;
            k += n;
            LC_CUDA(launch_residual_restrict<double>(s, c->op, c->psi(l), c->g(l), L.Nl[l], L.Pl[l], c->g(l + 1),
                                                     c->psi(l + 1), L.Pl[l + 1]));
        } else {
            LC_CUDA(launch_down<double>(s, tile_shape(c, l), c->op, c->psi(l), l > 0, c->g(l), c->psiB(l), L.Nl[l],
                                        L.Pl[l], c->g(l + 1), L.Pl[l + 1], c->nu1, c->beta));
        }
        ++k;
    }
    if (cluster_coarse(c, lc))
        LC_CUDA(launch_coarse_cluster<double>(s, c->op, c->g(lc), L.Pl[lc], c->psi(lc), L.Pl[lc], L.Nl[lc],
                                              vlevels(c) - lc, c->nu1, c->nu2, last_sweeps(c), c->beta, cluster_size(c),
                                              c->cluster_split));
    else
        LC_CUDA(launch_coarse<double>(s, c->op, c->g(lc), L.Pl[lc], lc == 0 ? c->psi(0) : nullptr, c->psi(lc),
                                      L.Pl[lc], L.Nl[lc], vlevels(c) - lc, c->nu1, c->nu2, last_sweeps(c), c->beta,
                                      lc == 0 ? rpart : nullptr, lc == 0 ? finish_args(c, 1, h) : kNoFinish));
    ++k;
    Correct64 none{nullptr, 0, nullptr, 0};
    for (int l = lc - 1; l >= 0; --l) {
        if (l < nph) {
            LC_CUDA(launch_prolong_correct<double>(s, c->psi(l), L.Nl[l], L.Pl[l], c->psi(l + 1), L.Pl[l + 1]));
            int n = level_sweeps(c, s, l, c->nu2);
            if (n < 0) return n;
            k += n;
        } else {
            LC_CUDA(launch_up<double>(s, tile_shape(c, l), c->op, c->psiB(l), c->g(l), c->psi(l + 1), L.Pl[l + 1],
                                      c->psi(l), L.Nl[l], L.Pl[l], c->nu2, c->beta, l == 0 ? rpart : nullptr, none,
                                      l == 0 ? finish_args(c, 0, h) : kNoFinish));
        }
        ++k;
    }
    *norm_done = lc == 0 || nph == 0;
    c->kernels_per_cycle = k;
    return LC_OK;
}

// Enqueues one mixed-precision refinement step: an FP32 V-cycle for the
// correction e of L_h e = r (r = the FP64 residual rounded to FP32, starting
// from e = 0), psi64 += e on the fine level, then the new FP64 residual with
// its norm partials (which also becomes the next step's r).
int enqueue_vcycle_mixed(lc_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    const Layout &L = c->lay;
    int lc = coarse_level(c);
    float beta = (float)c->beta;
    int k = 0;
    for (int l = 0; l < lc; ++l, ++k)
        LC_CUDA(launch_down<float>(s, tile_shape(c, l), c->op, nullptr, 1, c->g32(l), c->eB(l), L.Nl[l], L.Pl[l],
                                   c->g32(l + 1), L.Pl[l + 1], c->nu1, beta));
    if (cluster_coarse(c, lc))
        LC_CUDA(launch_coarse_cluster<float>(s, c->op, c->g32(lc), L.Pl[lc], c->eA(lc), L.Pl[lc], L.Nl[lc],
                                             vlevels(c) - lc, c->nu1, c->nu2, last_sweeps(c), beta, cluster_size(c),
                                             c->cluster_split));
    else
        LC_CUDA(launch_coarse<float>(s, c->op, c->g32(lc), L.Pl[lc], nullptr, c->eA(lc), L.Pl[lc], L.Nl[lc],
                                     vlevels(c) - lc, c->nu1, c->nu2, last_sweeps(c), beta, nullptr, kNoFinish));
    ++k;
    if (lc == 0) {
        LC_CUDA(launch_correct64(s, c->eA(0), L.Pl[0], c->psi(0), L.Pl[0], nullptr, L.Pl[0], c->N));
        ++k;
    }
    for (int l = lc - 1; l >= 0; --l, ++k) {
        Correct64 cor{nullptr, 0, nullptr, 0};
        if (l == 0) cor = Correct64{c->psi(0), L.Pl[0], nullptr, L.Pl[0]};
        LC_CUDA(launch_up<float>(s, tile_shape(c, l), c->op, c->eB(l), c->g32(l), c->eA(l + 1), L.Pl[l + 1], c->eA(l),
                                 L.Nl[l], L.Pl[l], c->nu2, beta, nullptr, cor, kNoFinish));
    }
    LC_CUDA(launch_residual64_to32(s, c->op, c->psi(0), c->g(0), c->N, L.Pl[0], c->at<float>(L.r32), L.Pl[0],
                                   c->at<double>(L.rpart), finish_args(c, L.nrpart_grid, h)));
    c->kernels_per_cycle = k + 1;
    return LC_OK;
}

// Body of one iteration of a Poisson loop: a cycle whose last kernel also
// computes the residual norm and takes the end-of-cycle decision (h != 0: the
// graph while-node's condition; h == 0: eager).
int enqueue_cycle_body(lc_ctx *c, cudaStream_t s, cudaGraphConditionalHandle h) {
    const Layout &L = c->lay;
    if (c->mixed()) return enqueue_vcycle_mixed(c, s, h);
    if (c->solver == 1) {  // one pass of sor_sweeps lexicographic sweeps, then the stopping test
        LC_CUDA(launch_sor_lex(s, c->op, c->psi(0), c->g(0), c->N, L.Pl[0], c->sor_sweeps, c->beta));
        LC_CUDA(launch_residual_norm<double>(s, c->op, c->psi(0), c->g(0), c->N, L.Pl[0], c->at<double>(L.rpart),
                                             finish_args(c, residual_norm64_blocks(c->N), h)));
        c->kernels_per_cycle = 2;
        return LC_OK;
    }
    bool norm_done = false;
    int rc = enqueue_vcycle(c, s, &norm_done, h);
    if (rc) return rc;
    if (!norm_done) {
        LC_CUDA(launch_residual_norm<double>(s, c->op, c->psi(0), c->g(0), c->N, L.Pl[0], c->at<double>(L.rpart),
                                             finish_args(c, residual_norm64_blocks(c->N), h)));
        c->kernels_per_cycle += 1;
    }
    return LC_OK;
}

// The five stages of one step, each: the fused L(omega) + stage combination,
// then a Poisson solve for the new stage vorticity.
struct StagePlan {
    double *in64, *out64;
    float *in32, *out32;
    StageCoef k;
};

void stage_plan(const lc_ctx *c, StagePlan st[5]) {
    const Layout &L = c->lay;
    double *W0 = c->at<double>(L.W0), *Wa = c->at<double>(L.Wa), *Wb = c->at<double>(L.Wb);
    float *W0s = c->mixed() ? c->at<float>(L.W0s) : nullptr, *Was = c->mixed() ? c->at<float>(L.Was) : nullptr,
          *Wbs = c->mixed() ? c->at<float>(L.Wbs) : nullptr;
    double dt = c->dt;
    st[0] = {W0, Wa, W0s, Was, StageCoef{1.0, 0.0, B10 * dt, 0.0, 0.0, 0}};
    st[1] = {Wa, Wb, Was, Wbs, StageCoef{A20, A21, B21 * dt, 0.0, 0.0, 0}};
    st[2] = {Wb, Wa, Wbs, Was, StageCoef{A30, A32, B32 * dt, A52, 0.0, 1}};
    st[3] = {Wa, Wb, Was, Wbs, StageCoef{A40, A43, B43 * dt, A53, B53 * dt, 2}};
    st[4] = {Wb, W0, Wbs, W0s, StageCoef{0.0, A54, B54 * dt, 0.0, 0.0, 3}};
}

// Mixed precision: the FP32 shadow of psi, read only by the next stage's
// L(omega), is refreshed once after each solve.
int enqueue_psi32(lc_ctx *c, cudaStream_t s) {
    if (!c->mixed() || c->rhs64) return LC_OK;
    const Layout &L = c->lay;
    LC_CUDA(launch_to32(s, c->psi(0), L.Pl[0], c->at<float>(L.psi32), L.Pl[0], c->N));
    return LC_OK;
}

int enqueue_thom(lc_ctx *c, cudaStream_t s) {
    const Layout &L = c->lay;
    if (c->mixed()) {
        double *w64[3] = {c->at<double>(L.W0), c->at<double>(L.Wa), c->at<double>(L.Wb)};
        float *w32[3] = {c->at<float>(L.W0s), c->at<float>(L.Was), c->at<float>(L.Wbs)};
        LC_CUDA(launch_thom_mixed(s, c->psi(0), w64, w32, c->N, L.Pl[0], L.Pl[0], c->U, c->profile));
    } else {
        LC_CUDA(launch_thom(s, c->psi(0), c->at<double>(L.W0), c->at<double>(L.Wa), c->at<double>(L.Wb), c->N,
                            L.Pl[0], c->U, c->profile));
    }
    return LC_OK;
}

// Everything of stage k before its Poisson loop.
int enqueue_stage_head(lc_ctx *c, cudaStream_t s, const StagePlan &st) {
    const Layout &L = c->lay;
    int N = c->N, P = L.Pl[0];
    if (c->mixed() && c->rhs64) {  // FP64 L(omega) from psi64; FP32 multigrid corrections
        LC_CUDA(launch_rhs_stage(s, c->psi(0), st.in64, c->at<double>(L.W0), c->at<double>(L.ACC), st.out64, N, P,
                                 c->Re, c->advect, st.k));
        LC_CUDA(launch_assemble_rhs(s, c->op, st.out64, c->g(0), N, P, c->at<double>(L.gpart)));
        LC_CUDA(launch_residual64_to32(s, c->op, c->psi(0), c->g(0), N, P, c->at<float>(L.r32), P,
                                       c->at<double>(L.rpart), kNoFinish));
    } else if (c->mixed()) {
        LC_CUDA(launch_rhs_stage_mixed(s, c->at<float>(L.psi32), P, st.in32, st.in64, c->at<double>(L.W0),
                                       c->at<double>(L.ACC), st.out64, st.out32, N, P, P, c->Re, c->advect, st.k));
        LC_CUDA(launch_assemble_rhs(s, c->op, st.out64, c->g(0), N, P, c->at<double>(L.gpart)));
        LC_CUDA(launch_residual64_to32(s, c->op, c->psi(0), c->g(0), N, P, c->at<float>(L.r32), P,
                                       c->at<double>(L.rpart), kNoFinish));
    } else {
        LC_CUDA(launch_rhs_stage(s, c->psi(0), st.in64, c->at<double>(L.W0), c->at<double>(L.ACC), st.out64, N, P,
                                 c->Re, c->advect, st.k));
        LC_CUDA(launch_assemble_rhs(s, c->op, st.out64, c->g(0), N, P, c->at<double>(L.gpart)));
    }
    return LC_OK;
}

// Captures one stage: head, the Poisson while-loop, Thom.
int capture_stage(lc_ctx *c, cudaStream_t s, const StagePlan &st) {
    int rc = enqueue_stage_head(c, s, st);
    if (rc) return rc;
    cudaStreamCaptureStatus cst;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    LC_CUDA(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphConditionalHandle h;
    LC_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    LC_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &p));
    cudaGraph_t body = p.conditional.phGraph_out[0];
    LC_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));

    LC_CUDA(cudaStreamBeginCaptureToGraph(c->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_cycle_body(c, c->cap2, h);
    cudaGraph_t tmp = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap2, &tmp);
    if (rc != LC_OK) return rc;
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture(body)");
    rc = enqueue_psi32(c, s);
    return rc ? rc : enqueue_thom(c, s);
}

// Eager mode: the same kernels launched one by one, the V-cycle loop driven
// from the host (one stream sync per cycle).  Used for per-kernel profiling:
// kernels inside a graph with conditional nodes cannot be profiled.
int eager_step(lc_ctx *c) {
    static const char *kStageName[5] = {"stage 1", "stage 2", "stage 3", "stage 4", "stage 5"};
    PdlScope pdl(c->pdl);
    cudaStream_t s = c->stream();
    StagePlan st[5];
    stage_plan(c, st);
    for (int k = 0; k < 5; ++k) {
        NvtxRange stage_range(kStageName[k]);
        int rc = enqueue_stage_head(c, s, st[k]);
        if (rc) return rc;
        for (;;) {
            NvtxRange cycle_range("poisson cycle");
            rc = enqueue_cycle_body(c, s, 0);
            if (rc) return rc;
            int more = 0;
            LC_CUDA(cudaMemcpyAsync(&more, &c->ds()->more, sizeof(int), cudaMemcpyDeviceToHost, s));
            LC_CUDA(cudaStreamSynchronize(s));
            if (!more) break;
        }
        rc = enqueue_psi32(c, s);
        if (rc == LC_OK) rc = enqueue_thom(c, s);
        if (rc) return rc;
    }
    return LC_OK;
}

int build_graph_once(lc_ctx *c);

// Builds the step graph.  If it cannot be captured or instantiated with
// programmatic-dependent-launch edges, it is built again without them; if the
// fused cooperative smoother is the obstacle, with one launch per colour
// phase.
int build_graph(lc_ctx *c) {
    int rc = LC_OK;
    for (int attempt = 0; attempt < 3; ++attempt) {
        {
            PdlScope pdl(c->pdl && !c->pdl_unsupported);
            rc = build_graph_once(c);
        }
        if (rc == LC_OK) break;
        cudaGetLastError();  // clear a launch error of the failed capture
        if (c->pdl && !c->pdl_unsupported) {
            c->pdl_unsupported = true;
        } else if (c->fused && (c->fused_blocks[0] || c->fused_blocks[1])) {
            c->fused_blocks[0] = c->fused_blocks[1] = 0;
        } else {
            break;
        }
    }
    return rc;
}

int build_graph_once(lc_ctx *c) {
    release_graph(c);
    StagePlan st[5];
    stage_plan(c, st);
    cudaStream_t s;
    LC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    int rc = LC_OK;
    for (int k = 0; k < 5 && rc == LC_OK; ++k) rc = capture_stage(c, s, st[k]);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (rc != LC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    c->graph = g;
    // per stage: L + combination, Poisson right-hand side, (mixed: first residual, psi shadow), Thom
    c->kernels_per_step = 5 * (c->mixed() ? (c->rhs64 ? 4 : 5) : 3);
    LC_CUDA(cudaGraphInstantiate(&c->exec, c->graph, 0));
    c->graph_dirty = false;
    return LC_OK;
}

int ensure_init(lc_ctx *c) {
    if (c->initialized) return LC_OK;
    LC_CUDA(cudaGetDevice(&c->device));
    LC_CUDA(init_mg_kernel_attributes());
    LC_CUDA(init_sor_kernel_attributes());
    c->fused_blocks[0] = smooth_fused_blocks(c->op, false);
    c->fused_blocks[1] = smooth_fused_blocks(c->op, true);
    if (!c->ws) {
        void *p = nullptr;
        LC_CUDA(cudaMalloc(&p, c->lay.total));
        c->ws = static_cast<char *>(p);
        c->ws_bytes = c->lay.total;
        c->ws_owned = true;
    }
    if (!c->own_stream) LC_CUDA(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    if (!c->cap2) LC_CUDA(cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking));
    cudaStream_t s = c->stream();
    LC_CUDA(cudaMemsetAsync(c->ws, 0, c->lay.total, s));
    int rc = enqueue_thom(c, s);
    if (rc) return rc;
    c->initialized = true;
    return LC_OK;
}

// Reads the device state after a stream sync and turns status bits into an error.
int sync_status(lc_ctx *c) {
    if (!c->initialized) return LC_OK;
    LC_CUDA(cudaStreamSynchronize(c->stream()));
    int status = 0;
    LC_CUDA(cudaMemcpy(&status, &c->ds()->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) {
        int zero = 0;
        LC_CUDA(cudaMemcpy(&c->ds()->status, &zero, sizeof(int), cudaMemcpyHostToDevice));
        if (status & kStatusNonFinite) return fail(LC_ERR_NONFINITE, "non-finite value in the Poisson residual or state");
        if (status & kStatusTimeout) {
            // a barrier that gave up left arrivals behind: start the next one from zero
            unsigned zero2[2] = {0u, 0u};
            LC_CUDA(cudaMemcpy(&c->ds()->bar_count, zero2, sizeof(zero2), cudaMemcpyHostToDevice));
            return fail(LC_ERR_TIMEOUT, "a device-side grid barrier wait gave up");
        }
        if (status & kStatusNoConv) return fail(LC_ERR_NOCONV, "a Poisson solve reached max_cycles above tol");
    }
    return LC_OK;
}

int copy_field_out(lc_ctx *c, size_t off, double *host, size_t n) {
    size_t need = (size_t)(c->N + 1) * (c->N + 1);
    if (!host) return fail(LC_ERR_ARG, "NULL host buffer");
    if (n < need) return fail(LC_ERR_SIZE, "host buffer smaller than (N+1)^2");
    int rc = ensure_init(c);
    if (rc) return rc;
    LC_CUDA(cudaMemcpy2DAsync(host, (c->N + 1) * sizeof(double), c->at<double>(off), c->lay.Pl[0] * sizeof(double),
                              (c->N + 1) * sizeof(double), c->N + 1, cudaMemcpyDeviceToHost, c->stream()));
    return sync_status(c);
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

lc_ctx *lc_create(int N, double Re, double dt, double tol) {
    if (!valid_N(N)) {
        fail(LC_ERR_ARG, "N must be 2^k, 3*2^k, 5*2^k or 7*2^k with 8 <= N <= 8192");
        return nullptr;
    }
    if (!(Re > 0.0) || !std::isfinite(Re) || !(tol > 0.0) || !std::isfinite(dt)) {
        fail(LC_ERR_ARG, "Re and tol must be positive and finite");
        return nullptr;
    }
    double h = 1.0 / N;
    if (dt <= 0.0) dt = 0.25 * std::fmin(h, Re * h * h / 4.0);
    lc_ctx *c = new lc_ctx();
    c->N = N;
    c->Re = Re;
    c->dt = dt;
    c->tol = tol;
    make_layout(N, c->precision, c->lay);
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live.insert(c);
    }
    g_err.clear();
    return c;
}

void lc_destroy(lc_ctx *c) {
    if (!live(c)) return;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live.erase(c);
    }
    if (c->initialized) cudaStreamSynchronize(c->stream());
    release_graph(c);
    if (c->ws_owned && c->ws) cudaFree(c->ws);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->cap2) cudaStreamDestroy(c->cap2);
    delete c;
}

const char *lc_last_error(void) { return g_err.c_str(); }

size_t lc_workspace_bytes(int N, int precision) {
    Layout L;
    return make_layout(N, precision, L) ? L.total : 0;
}

int lc_bind_workspace(lc_ctx *c, void *dev_ptr, size_t bytes) {
    LC_CHECK_CTX(c);
    if (c->initialized) return fail(LC_ERR_ARG, "workspace must be bound before first use");
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255)) return fail(LC_ERR_SIZE, "workspace must be 256-byte aligned");
    if (bytes < c->lay.total) return fail(LC_ERR_SIZE, "workspace smaller than lc_workspace_bytes");
    c->ws = static_cast<char *>(dev_ptr);
    c->ws_bytes = bytes;
    c->ws_owned = false;
    return LC_OK;
}

int lc_set_stream(lc_ctx *c, void *stream) {
    LC_CHECK_CTX(c);
    if (c->initialized) {
        // order the old stream's work before anything on the new one
        cudaEvent_t ev;
        LC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        LC_CUDA(cudaEventRecord(ev, c->stream()));
        c->user_stream = static_cast<cudaStream_t>(stream);
        c->use_user_stream = true;
        LC_CUDA(cudaStreamWaitEvent(c->stream(), ev, 0));
        LC_CUDA(cudaEventDestroy(ev));
    } else {
        c->user_stream = static_cast<cudaStream_t>(stream);
        c->use_user_stream = true;
    }
    return LC_OK;
}

int lc_set_option(lc_ctx *c, const char *key, double v) {
    LC_CHECK_CTX(c);
    if (!key) return fail(LC_ERR_ARG, "NULL option key");
    std::string k(key);
    int iv = (int)v;
    bool integral = v == (double)iv;
    if (k == "op") {
        if (c->initialized) return fail(LC_ERR_ARG, "op must be set before first use");
        if (!integral || (iv != LC_OP_5PT && iv != LC_OP_COMPACT)) return fail(LC_ERR_ARG, "op must be 0 or 1");
        c->op = iv;
    } else if (k == "precision") {
        if (c->initialized) return fail(LC_ERR_ARG, "precision must be set before first use");
        if (!integral || (iv != LC_PREC_FP64 && iv != LC_PREC_MIXED)) return fail(LC_ERR_ARG, "precision must be 0 or 1");
        if (iv == LC_PREC_MIXED && c->solver == 1) return fail(LC_ERR_ARG, "the SOR solver runs in FP64 precision only");
        c->precision = iv;
        make_layout(c->N, c->precision, c->lay);
    } else if (k == "nu1" || k == "nu2") {
        if (!integral || iv < 1 || iv > 16) return fail(LC_ERR_ARG, "nu1/nu2 must be 1..16");
        (k == "nu1" ? c->nu1 : c->nu2) = iv;
    } else if (k == "nuc") {
        if (!integral || iv < 1 || iv > 256) return fail(LC_ERR_ARG, "nuc must be 1..256");
        c->nuc = iv;
    } else if (k == "beta") {
        if (!(v > 0.0 && v < 2.0)) return fail(LC_ERR_ARG, "beta must be in (0, 2)");
        c->beta = v;
    } else if (k == "solver") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "solver must be 0 (multigrid) or 1 (SOR)");
        if (iv == 1 && c->mixed()) return fail(LC_ERR_ARG, "the SOR solver runs in FP64 precision only");
        c->solver = iv;
    } else if (k == "coarse_direct") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "coarse_direct must be 0 or 1");
        c->coarse_direct = iv;
    } else if (k == "rhs64") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "rhs64 must be 0 or 1");
        c->rhs64 = iv;
    } else if (k == "barrier_extra") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "barrier_extra must be 0 or 1");
        c->barrier_extra = iv;
    } else if (k == "fused") {
        if (!integral || iv < 0 || iv > 3) return fail(LC_ERR_ARG, "fused must be 0..3");
        c->fused = iv;
    } else if (k == "sor_sweeps") {
        if (!integral || iv < 1 || iv > 4096) return fail(LC_ERR_ARG, "sor_sweeps must be 1..4096");
        c->sor_sweeps = iv;
    } else if (k == "max_cycles") {
        if (!integral || iv < 1) return fail(LC_ERR_ARG, "max_cycles must be >= 1");
        c->max_cycles = iv;
    } else if (k == "U" || k == "profile") {
        if (k == "U") {
            if (!std::isfinite(v)) return fail(LC_ERR_ARG, "U must be finite");
            c->U = v;
        } else {
            if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "profile must be 0 or 1");
            c->profile = iv;
        }
        if (c->initialized) {
            int rc = enqueue_thom(c, c->stream());
            if (rc) return rc;
        }
    } else if (k == "advect") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "advect must be 0 or 1");
        c->advect = iv;
    } else if (k == "fine_phases") {
        if (!integral || iv < 0 || iv > kMaxLevels) return fail(LC_ERR_ARG, "fine_phases must be 0..16");
        c->fine_phases = iv;
    } else if (k == "blocked") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, k + " must be 0 or 1");
        c->blocked = iv;
    } else if (k == "tile_shape") {
        if (!integral || iv < -1 || iv > 4) return fail(LC_ERR_ARG, "tile_shape must be -1 (auto) or 0..4");
        c->tile_force = iv;
    } else if (k == "coarse_max") {
        if (!integral || iv < 2 || iv > 256) return fail(LC_ERR_ARG, "coarse_max must be 2..256");
        c->coarse_max = iv;
    } else if (k == "pdl") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "pdl must be 0 or 1");
        c->pdl = iv;
        c->pdl_unsupported = false;
    } else if (k == "coarse_cluster") {
        if (!integral || iv < -1 || iv == 1 || iv > 16)
            return fail(LC_ERR_ARG, "coarse_cluster must be -1 (auto), 0 (off) or 2..16");
        c->coarse_cluster = iv;
    } else if (k == "cluster_max") {
        if (!integral || iv < 8 || iv > 512) return fail(LC_ERR_ARG, "cluster_max must be 8..512");
        c->cluster_max = iv;
    } else if (k == "cluster_split") {
        if (!integral || iv < 4 || iv > 256) return fail(LC_ERR_ARG, "cluster_split must be 4..256");
        c->cluster_split = iv;
    } else if (k == "graph") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "graph must be 0 or 1");
        c->use_graph = iv;
        return LC_OK;
    } else if (k == "monitor") {
        if (!integral || (iv != 0 && iv != 1)) return fail(LC_ERR_ARG, "monitor must be 0 or 1");
        c->monitor = iv;
        return LC_OK;
    } else {
        return fail(LC_ERR_ARG, "unknown option " + k);
    }
    c->graph_dirty = true;
    return LC_OK;
}

int lc_step(lc_ctx *c, int nsteps) {
    LC_CHECK_CTX(c);
    if (nsteps < 0) return fail(LC_ERR_ARG, "nsteps must be >= 0");
    NvtxRange range("lc_step");
    int rc = ensure_init(c);
    if (rc) return rc;
    if (c->use_graph && c->graph_dirty) {
        rc = build_graph(c);
        if (rc) return rc;
    }
    cudaStream_t s = c->stream();
    const Layout &L = c->lay;
    size_t rowb = (size_t)L.Pl[0] * sizeof(double), fb = rowb * (c->N + 1);
    for (int n = 0; n < nsteps; ++n) {
        bool last = n == nsteps - 1;
        if (last && c->monitor) {
            LC_CUDA(cudaMemcpyAsync(c->at<double>(L.snap_psi), c->psi(0), fb, cudaMemcpyDeviceToDevice, s));
            LC_CUDA(cudaMemcpyAsync(c->at<double>(L.snap_w), c->at<double>(L.W0), fb, cudaMemcpyDeviceToDevice, s));
        }
        if (c->use_graph) {
            LC_CUDA(cudaGraphLaunch(c->exec, s));
        } else {
            rc = eager_step(c);
            if (rc) return rc;
        }
        if (last && c->monitor) {
            LC_CUDA(launch_monitor(s, c->at<double>(L.snap_psi), c->psi(0), c->at<double>(L.snap_w),
                                   c->at<double>(L.W0), c->N, L.Pl[0], c->at<double>(L.mpart), c->ds(), c->dt));
            c->mon_valid = true;
        }
        c->steps++;
    }
    return LC_OK;
}

int lc_get_psi(lc_ctx *c, double *host, size_t n) {
    LC_CHECK_CTX(c);
    return copy_field_out(c, c->lay.psi[0], host, n);
}

int lc_get_omega(lc_ctx *c, double *host, size_t n) {
    LC_CHECK_CTX(c);
    return copy_field_out(c, c->lay.W0, host, n);
}

double lc_residual(lc_ctx *c) {
    if (!live(c)) {
        fail(LC_ERR_ARG, "invalid context");
        return NAN;
    }
    // device errors stay pending for the next int-returning call
    if (ensure_init(c) != LC_OK || cudaStreamSynchronize(c->stream()) != cudaSuccess) return NAN;
    double rel = 0.0;
    if (cudaMemcpy(&rel, &c->ds()->last_rel, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return NAN;
    return rel;
}

int lc_synchronize(lc_ctx *c) {
    LC_CHECK_CTX(c);
    return sync_status(c);
}

int lc_monitor(lc_ctx *c, double out[4]) {
    LC_CHECK_CTX(c);
    if (!out) return fail(LC_ERR_ARG, "NULL output");
    int rc = ensure_init(c);
    if (rc) return rc;
    rc = sync_status(c);
    DevState head;
    LC_CUDA(cudaMemcpy(&head, c->ds(), offsetof(DevState, log), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) out[k] = c->mon_valid ? head.mon[k] : 0.0;
    out[3] = head.last_cycles;
    return rc;
}

int lc_set_state(lc_ctx *c, const double *psi, const double *omega) {
    LC_CHECK_CTX(c);
    if (!psi || !omega) return fail(LC_ERR_ARG, "NULL state array");
    int rc = ensure_init(c);
    if (rc) return rc;
    cudaStream_t s = c->stream();
    const Layout &L = c->lay;
    size_t hp = (c->N + 1) * sizeof(double), dp = L.Pl[0] * sizeof(double);
    LC_CUDA(cudaMemcpy2DAsync(c->psi(0), dp, psi, hp, hp, c->N + 1, cudaMemcpyHostToDevice, s));
    LC_CUDA(launch_zero_walls(s, c->psi(0), c->N, L.Pl[0]));
    LC_CUDA(cudaMemcpy2DAsync(c->at<double>(L.W0), dp, omega, hp, hp, c->N + 1, cudaMemcpyHostToDevice, s));
    if (c->mixed()) {
        LC_CUDA(launch_to32(s, c->psi(0), L.Pl[0], c->at<float>(L.psi32), L.Pl[0], c->N));
        LC_CUDA(launch_to32(s, c->at<double>(L.W0), L.Pl[0], c->at<float>(L.W0s), L.Pl[0], c->N));
    }
    rc = enqueue_thom(c, s);
    if (rc) return rc;
    LC_CUDA(cudaStreamSynchronize(s));  // the host arrays may be released on return
    return LC_OK;
}

int lc_cycle_log(lc_ctx *c, int *out, size_t max, size_t *n_out) {
    LC_CHECK_CTX(c);
    if (!out || !n_out) return fail(LC_ERR_ARG, "NULL output");
    int rc = ensure_init(c);
    if (rc) return rc;
    rc = sync_status(c);
    DevState head;
    LC_CUDA(cudaMemcpy(&head, c->ds(), offsetof(DevState, log), cudaMemcpyDeviceToHost));
    std::vector<int> ring(kLogN);
    LC_CUDA(cudaMemcpy(ring.data(), c->ds()->log, sizeof(int) * kLogN, cudaMemcpyDeviceToHost));
    unsigned long long total = head.nsolves, avail = total < (unsigned long long)kLogN ? total : kLogN;
    size_t n = avail < max ? (size_t)avail : max;
    for (size_t k = 0; k < n; ++k) out[k] = ring[(total - avail + k) % kLogN];
    *n_out = n;
    return rc;
}

int lc_get_params(lc_ctx *c, double out[7]) {
    LC_CHECK_CTX(c);
    if (!out) return fail(LC_ERR_ARG, "NULL output");
    out[0] = c->N;
    out[1] = c->Re;
    out[2] = c->dt;
    out[3] = c->tol;
    out[4] = 1.0 / c->N;
    out[5] = vlevels(c);
    out[6] = (double)c->steps;
    return LC_OK;
}

int lc_selftest_conversions(long long n, unsigned long long seed, long long mismatches[2]) {
    if (n < 0 || !mismatches) return fail(LC_ERR_ARG, "n must be >= 0 and mismatches non-NULL");
    int dev = 0;
    LC_CUDA(cudaGetDevice(&dev));
    cudaStream_t s;
    LC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    unsigned long long *bad = nullptr, h[2] = {0, 0};
    cudaError_t e = cudaMalloc(&bad, sizeof(h));
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(h), s);
    if (e == cudaSuccess) e = launch_selftest_conversions(s, n, seed, bad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, bad, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (bad) cudaFree(bad);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return cuda_fail(e, "lc_selftest_conversions");
    mismatches[0] = (long long)h[0];
    mismatches[1] = (long long)h[1];
    return LC_OK;
}

int lc_launch_stats(lc_ctx *c, double out[2]) {
    LC_CHECK_CTX(c);
    if (!out) return fail(LC_ERR_ARG, "NULL output");
    if (c->graph_dirty) {
        int rc = ensure_init(c);
        if (rc == LC_OK) rc = build_graph(c);
        if (rc) return rc;
    }
    out[0] = c->kernels_per_step + (c->monitor ? 1 : 0);  // the same kernels in graph and eager mode
    out[1] = c->kernels_per_cycle;
    return LC_OK;
}

int lc_bench_kernel(lc_ctx *c, int kernel, int reps, double out[4]) {
    LC_CHECK_CTX(c);
    int nk = c->mixed() ? 4 : 5;
    if (!out || reps < 1 || kernel < 0 || kernel >= nk) return fail(LC_ERR_ARG, "bad kernel id, reps or output");
    int rc = ensure_init(c);
    if (rc) return rc;
    cudaStream_t s = c->stream();
    const Layout &L = c->lay;
    int N = c->N, P = L.Pl[0];
    double n_int = (double)(N - 1) * (N - 1), n_c = (double)(N / 2 - 1) * (N / 2 - 1);
    int ncol = c->op == LC_OP_COMPACT ? 4 : 2;
    double sw_flops = c->op == LC_OP_COMPACT ? 10.0 : 5.0;  // per node per sweep: 6 adds + 2 FMAs (5-point: 3 + 1)
    double res_flops = sw_flops + 1.0;
    StageCoef k2{A20, A21, B21 * c->dt, 0.0, 0.0, 0};
    auto launch = [&](int r) -> cudaError_t {
        if (!c->mixed()) {
            switch (kernel) {
                case 0:
                    return launch_smooth_colour<double>(s, c->op, c->psi(0), c->g(0), N, P, r % ncol, c->beta);
                case 1:
                    return launch_rhs_stage(s, c->psi(0), c->at<double>(L.Wa), c->at<double>(L.W0),
                                            c->at<double>(L.ACC), c->at<double>(L.Wb), N, P, c->Re, c->advect, k2);
                case 2:
                    return launch_residual_restrict<double>(s, c->op, c->psi(0), c->g(0), N, P, c->g(1), c->psi(1),
                                                            L.Pl[1]);
                case 3:
                    return launch_sor_lex(s, c->op, c->psi(0), c->g(0), N, P, c->sor_sweeps, c->beta);
                default:
                    return launch_smooth_fused<double>(s, c->op, c->psi(0), c->g(0), N, P, c->nu1, c->beta, c->ds(),
                                                       c->fused_blocks[c->beta != 1.0 ? 1 : 0], c->barrier_extra);
            }
        }
        switch (kernel) {
            case 0:
                return launch_down<float>(s, tile_shape(c, 0), c->op, nullptr, 1, c->g32(0), c->eB(0), N, P, c->g32(1),
                                          L.Pl[1], c->nu1, (float)c->beta);
            case 1:
                if (c->rhs64)
                    return launch_rhs_stage(s, c->psi(0), c->at<double>(L.Wa), c->at<double>(L.W0),
                                            c->at<double>(L.ACC), c->at<double>(L.Wb), N, P, c->Re, c->advect, k2);
                return launch_rhs_stage_mixed(s, c->at<float>(L.psi32), P, c->at<float>(L.Was), c->at<double>(L.Wa),
                                              c->at<double>(L.W0), c->at<double>(L.ACC), c->at<double>(L.Wb),
                                              c->at<float>(L.Wbs), N, P, P, c->Re, c->advect, k2);
            case 2:
                return launch_residual64_to32(s, c->op, c->psi(0), c->g(0), N, P, c->at<float>(L.r32), P,
                                              c->at<double>(L.rpart), kNoFinish);
            default: {
                Correct64 cor{c->psi(0), P, nullptr, P};
                return launch_up<float>(s, tile_shape(c, 0), c->op, c->eB(0), c->g32(0), c->eA(1), L.Pl[1], c->eA(0), N,
                                        P, c->nu2, (float)c->beta, nullptr, cor, kNoFinish);
            }
        }
    };
    if (c->mixed() && (kernel == 0 || kernel == 3) && coarse_level(c) == 0)
        return fail(LC_ERR_ARG, "grid too small for the tile kernels");
    if (!c->mixed() && kernel == 4 && !c->fused_blocks[c->beta != 1.0 ? 1 : 0])
        return fail(LC_ERR_ARG, "the fused smoother is not available on this device");
    cudaEvent_t e0, e1;
    LC_CUDA(cudaEventCreate(&e0));
    LC_CUDA(cudaEventCreate(&e1));
    LC_CUDA(launch(0));  // warm the instruction cache
    LC_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) LC_CUDA(launch(r));
    LC_CUDA(cudaEventRecord(e1, s));
    LC_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    LC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out[0] = ms / reps;
    out[2] = out[3] = 0.0;
    if (!c->mixed()) {
        switch (kernel) {
            case 0: {  // read psi once, read g and write psi at the colour's nodes
                double nc = n_int / ncol;
                out[1] = 8.0 * n_int + 16.0 * nc;
                out[2] = (sw_flops + (c->beta != 1.0 ? 3.0 : 0.0)) * nc;
                break;
            }
            case 1:  // stage 2: read omega^(1), psi, omega^n; write omega^(2)
                out[1] = 32.0 * n_int;
                out[2] = (c->advect ? 27.0 : 13.0) * n_int;
                break;
            case 2:  // read psi, g; write the coarse g and zero the coarse psi
                out[1] = 16.0 * n_int + 16.0 * n_c;
                out[2] = res_flops * n_int + 8.0 * n_c;
                break;
            case 3:  // sor_sweeps sweeps; the grid is read and written once per launch
                out[1] = 24.0 * n_int;
                out[2] = c->sor_sweeps * (sw_flops + (c->beta != 1.0 ? 3.0 : 0.0)) * n_int;
                break;
            default:  // nu1 colour sweeps: psi and g read once, psi written once
                out[1] = 24.0 * n_int;
                out[2] = c->nu1 * (sw_flops + (c->beta != 1.0 ? 3.0 : 0.0)) * n_int;
        }
    } else {
        switch (kernel) {
            case 0:  // read r32; write e32 and the coarse g32; nu1 sweeps + residual + restriction in FP32
                out[1] = 8.0 * n_int + 4.0 * n_c;
                out[3] = (c->nu1 * sw_flops + res_flops) * n_int + 8.0 * n_c;
                break;
            case 1:
                if (c->rhs64) {  // as the FP64 path: read omega^(1), psi, omega^n; write omega^(2)
                    out[1] = 32.0 * n_int;
                    out[2] = (c->advect ? 27.0 : 13.0) * n_int;
                } else {  // read omega32 (stencil), psi32, omega64, W0; write omega64 and its shadow
                    out[1] = 36.0 * n_int;
                    out[2] = 5.0 * n_int;
                    out[3] = (c->advect ? 22.0 : 8.0) * n_int;
                }
                break;
            case 2:  // read psi64, g64; write r32
                out[1] = 20.0 * n_int;
                out[2] = (res_flops + 1.0) * n_int;
                break;
            default:  // read e32, r32, coarse e, psi64; write psi64
                out[1] = 24.0 * n_int + 4.0 * n_c;
                out[2] = 1.0 * n_int;
                out[3] = (c->nu2 * sw_flops + 3.0) * n_int;
        }
    }
    return LC_OK;
}

struct CkptHeader {
    char magic[4];
    int version, N, precision, op, pad;
    double Re, dt, tol, U;
    long long steps;
};

int lc_save(lc_ctx *c, const char *path) {
    LC_CHECK_CTX(c);
    if (!path) return fail(LC_ERR_ARG, "NULL path");
    size_t n = (size_t)(c->N + 1) * (c->N + 1);
    std::vector<double> psi(n), w(n);
    int rc = lc_get_psi(c, psi.data(), n);
    if (rc) return rc;
    rc = lc_get_omega(c, w.data(), n);
    if (rc) return rc;
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "LCCK", 4);
    h.version = 1;
    h.N = c->N;
    h.precision = c->precision;
    h.op = c->op;
    h.Re = c->Re;
    h.dt = c->dt;
    h.tol = c->tol;
    h.U = c->U;
    h.steps = c->steps;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(LC_ERR_IO, std::string("cannot open ") + path);
    bool ok = fwrite(&h, sizeof(h), 1, f) == 1 && fwrite(psi.data(), sizeof(double), n, f) == n &&
              fwrite(w.data(), sizeof(double), n, f) == n;
    ok = (fclose(f) == 0) && ok;
    return ok ? LC_OK : fail(LC_ERR_IO, "short write");
}

int lc_load(lc_ctx *c, const char *path) {
    LC_CHECK_CTX(c);
    if (!path) return fail(LC_ERR_ARG, "NULL path");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(LC_ERR_IO, std::string("cannot open ") + path);
    CkptHeader h;
    bool ok = fread(&h, sizeof(h), 1, f) == 1 && !memcmp(h.magic, "LCCK", 4) && h.version == 1;
    if (!ok || h.N != c->N) {
        fclose(f);
        return fail(LC_ERR_IO, "not a checkpoint of this grid size");
    }
    size_t n = (size_t)(c->N + 1) * (c->N + 1);
    std::vector<double> psi(n), w(n);
    ok = fread(psi.data(), sizeof(double), n, f) == n && fread(w.data(), sizeof(double), n, f) == n;
    fclose(f);
    if (!ok) return fail(LC_ERR_IO, "truncated checkpoint");
    int rc = lc_set_state(c, psi.data(), w.data());
    if (rc == LC_OK) c->steps = h.steps;
    return rc;
}

}  // extern "C"
