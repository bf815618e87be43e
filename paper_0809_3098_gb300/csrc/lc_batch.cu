// Batched engine: many lid-driven cavities of different sizes and Reynolds
// numbers advanced together, one CUDA graph launch per SSPRK(5,4) step.
//
// Every cavity runs the mixed-precision step of the single-cavity library
// (FP32 multigrid correction cycles inside an FP64 residual / refinement
// loop, FP32 L(omega) with FP64 stage accumulation, FP64 Thom; method of
// Cardoso & Bicudo, arXiv:0809.3098, Secs. 2-3).  Each kernel launch covers
// the work of all cavities: a table of per-cavity block ranges maps a block to
// its cavity and tile.  Each cavity keeps its own stopping rule: when it
// converges its blocks go idle, and the graph's while-node repeats the cycle
// while any cavity still iterates, so every cavity makes exactly the cycles it
// would make alone (and gives the same bits).
#include "lc_internal.h"

#include "../../include/lc.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

using namespace lcx;

namespace {

std::mutex g_bmu;
std::set<const void *> g_blive;

int bfail(int code, const std::string &msg) {
    set_last_error(msg.c_str());
    return code;
}

int bcuda(cudaError_t e, const char *what) {
    return bfail(LC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bcuda(e_, #call);    \
    } while (0)

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
int pitch32(int N) { return ((N + 1 + 31) / 32) * 32; }

int nlevels(int N) {
    int n = 1;
    while (N % 2 == 0 && N >= 4) {
        N /= 2;
        ++n;
    }
    return (N == 2 || N == 3 || N == 5 || N == 7) ? n : -1;
}

constexpr int kSBX = 32, kSBY = 8;  // stage-kernel block
constexpr int kResRange = 1 + kMaxLevels;  // index of the residual kernels' block range

struct BLayout {
    std::vector<size_t> psi64, g64, psi32, W[4], Ws[3], log;
    std::vector<std::vector<size_t>> eA, eB, g32;
    size_t cav, ranges, state, rpart, gpart, total;
    int nranges, stage_blocks;
};

}  // namespace

struct lc_batch {
    int count = 0;
    std::vector<int> N, nlev, lc;
    std::vector<int> nv;  // levels the V-cycle visits (the last one solved exactly with coarse_direct)
    int coarse_direct = 1;
    std::vector<double> Re, dt;
    double tol = 1e-10, beta = 1.1, U = 1.0;
    int op = LC_OP_COMPACT, nu1 = 2, nu2 = 1, nuc = 16, max_cycles = 100, advect = 1, coarse_max = 64;
    int use_graph = 1, rhs64 = 1;  // rhs64: L(omega) in FP64 (0: from the FP32 shadows)
    int pdl = 1;                   // programmatic dependent launch of the step's kernels
    bool pdl_unsupported = false;  // a graph with PDL edges failed to build
    int Lmax = 0;
    std::vector<int> shape;  // tile shape per level (< Lmax)

    BLayout lay;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false, initialized = false;
    std::vector<BatchCav> hcav;
    std::vector<BatchRange> hr;  // [0] stage range, [1 + l] level-l tile range
    std::vector<int> rblocks;
    size_t coarse_smem = 0;

    cudaStream_t own = nullptr, user = nullptr, cap2 = nullptr;
    bool use_user = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;
    long long steps = 0;

    cudaStream_t stream() const { return use_user ? user : own; }
    template <typename T>
    T *at(size_t off) const {
        return reinterpret_cast<T *>(ws + off);
    }
    BatchCav *dcav() const { return at<BatchCav>(lay.cav); }
    BatchRange *drange(int k) const { return at<BatchRange>(lay.ranges) + k; }
    BatchState *dstate() const { return at<BatchState>(lay.state); }
};

namespace {

bool blive(const lc_batch *b) {
    std::lock_guard<std::mutex> lk(g_bmu);
    return b && g_blive.count(b);
}

#define LB_CHECK(b)                                                        \
    do {                                                                   \
        if (!blive(b)) return bfail(LC_ERR_ARG, "invalid batch context"); \
    } while (0)

int coarse_level_of(int N, int nl, int cmax) {
    for (int l = 0; l < nl; ++l)
        if ((N >> l) <= cmax && coarse_smem_bytes(N >> l, nl - l, 4) <= kMaxSmem - 1024) return l;
    return nl - 1;
}

int stage_blocks_of(int N) { return ((N - 1 + kSBX - 1) / kSBX) * ((N - 1 + kSBY - 1) / kSBY); }

// Workspace layout and the host copies of the descriptors and block ranges.
bool plan(lc_batch *b) {
    BLayout &L = b->lay;
    L = BLayout();
    int C = b->count;
    b->nlev.assign(C, 0);
    b->nv.assign(C, 0);
    b->lc.assign(C, 0);
    b->Lmax = 0;
    for (int c = 0; c < C; ++c) {
        b->nlev[c] = nlevels(b->N[c]);
        b->nv[c] = b->nlev[c];
        if (b->coarse_direct)  // the first level below the fine one with at most 16 intervals is solved exactly
            for (int l = 1; l < b->nlev[c]; ++l)
                if ((b->N[c] >> l) <= 16) {
                    b->nv[c] = l + 1;
                    break;
                }
        b->lc[c] = coarse_level_of(b->N[c], b->nv[c], b->coarse_max);
        if (b->lc[c] < 1) return false;  // every cavity has at least one tile level
        if (b->lc[c] > b->Lmax) b->Lmax = b->lc[c];
    }
    if ((int)b->shape.size() != b->Lmax) b->shape.assign(b->Lmax, -1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += al256(bytes);
        return o;
    };
    L.eA.assign(C, {});
    L.eB.assign(C, {});
    L.g32.assign(C, {});
    for (int k = 0; k < 4; ++k) L.W[k].assign(C, 0);
    for (int k = 0; k < 3; ++k) L.Ws[k].assign(C, 0);
    L.psi64.assign(C, 0);
    L.g64.assign(C, 0);
    L.psi32.assign(C, 0);
    L.log.assign(C, 0);
    b->hcav.assign(C, BatchCav());
    b->coarse_smem = 0;
    for (int c = 0; c < C; ++c) {
        int N = b->N[c];
        size_t n0 = (size_t)(N + 1) * pitch32(N);
        L.psi64[c] = take(n0 * 8);
        L.g64[c] = take(n0 * 8);
        L.psi32[c] = take(n0 * 4);
        for (int k = 0; k < 4; ++k) L.W[k][c] = take(n0 * 8);
        for (int k = 0; k < 3; ++k) L.Ws[k][c] = take(n0 * 4);
        L.eA[c].assign(b->nlev[c], 0);
        L.eB[c].assign(b->nlev[c], 0);
        L.g32[c].assign(b->nlev[c], 0);
        for (int l = 0; l < b->nlev[c]; ++l) {
            int n = N >> l;
            size_t m = (size_t)(n + 1) * pitch32(n) * 4;
            L.eA[c][l] = take(m);
            L.eB[c][l] = take(m);
            L.g32[c][l] = take(m);  // level 0: the FP32 residual
        }
        L.log[c] = take(sizeof(int) * kLogN);
        int cl = b->lc[c];
        size_t cs = coarse_smem_bytes(N >> cl, b->nv[c] - cl, 4);
        if (cs > b->coarse_smem) b->coarse_smem = cs;
    }
    L.nranges = 2 + kMaxLevels;  // [0] stage, [1 + l] level-l tiles, [kResRange] residual
    L.cav = take(sizeof(BatchCav) * C);
    L.ranges = take(sizeof(BatchRange) * L.nranges);  // independent of the options
    L.state = take(sizeof(BatchState));
    int sb = 0, rb = 0;
    for (int c = 0; c < C; ++c) {
        sb += stage_blocks_of(b->N[c]);
        rb += residual_norm_blocks(b->N[c]);
    }
    L.stage_blocks = sb;
    L.rpart = take(sizeof(double) * rb);
    L.gpart = take(sizeof(double) * sb);
    L.total = off;
    return true;
}

int shape_of(const lc_batch *b, int l) {
    int nu = b->nu1 > b->nu2 ? b->nu1 : b->nu2;
    int nmax = 0;
    for (int c = 0; c < b->count; ++c)
        if (l < b->lc[c] && (b->N[c] >> l) > nmax) nmax = b->N[c] >> l;
    return tile_shape_for(nmax, b->op, nu, 4, b->shape[l]);
}

// Fills the device descriptors and block ranges (workspace must be set).
void fill_tables(lc_batch *b) {
    const BLayout &L = b->lay;
    int C = b->count;
    for (int c = 0; c < C; ++c) {
        BatchCav &v = b->hcav[c];
        int keep_active = v.active;
        memset(&v, 0, sizeof(v));
        v.active = keep_active;
        v.N = b->N[c];
        v.nlev = b->nv[c];
        v.lc = b->lc[c];
        for (int l = 0; l < b->nlev[c]; ++l) {
            v.P[l] = pitch32(v.N >> l);
            v.eA[l] = b->at<float>(L.eA[c][l]);
            v.eB[l] = b->at<float>(L.eB[c][l]);
            v.g32[l] = b->at<float>(L.g32[c][l]);
        }
        v.Re = b->Re[c];
        v.dt = b->dt[c];
        double h = 1.0 / v.N;
        v.h2 = h * h;
        v.nu_invh2 = (double)v.N * (double)v.N / v.Re;
        v.nu_invh2f = (float)((double)v.N * (double)v.N / v.Re);
        v.psi64 = b->at<double>(L.psi64[c]);
        v.g64 = b->at<double>(L.g64[c]);
        v.psi32 = b->at<float>(L.psi32[c]);
        for (int k = 0; k < 4; ++k) v.W[k] = b->at<double>(L.W[k][c]);
        for (int k = 0; k < 3; ++k) v.Ws[k] = b->at<float>(L.Ws[k][c]);
        v.log = b->at<int>(L.log[c]);
    }
    b->hr.assign(L.nranges, BatchRange());
    b->rblocks.assign(L.nranges, 0);
    // stage range: every cavity, 32 x 8 node blocks
    {
        BatchRange &r = b->hr[0];
        r.count = C;
        int s = 0;
        for (int c = 0; c < C; ++c) {
            r.start[c] = s;
            r.gx[c] = (b->N[c] - 1 + kSBX - 1) / kSBX;
            s += stage_blocks_of(b->N[c]);
        }
        r.start[C] = s;
        b->rblocks[0] = s;
    }
    // residual range: every cavity, blocks of kRX x kRY interior nodes
    {
        BatchRange &r = b->hr[kResRange];
        r.count = C;
        int s = 0;
        for (int c = 0; c < C; ++c) {
            r.start[c] = s;
            r.gx[c] = residual_blocks_x(b->N[c]);
            s += residual_norm_blocks(b->N[c]);
        }
        r.start[C] = s;
        b->rblocks[kResRange] = s;
    }
    // level-l tile ranges: cavities whose level l is a tile level (l < lc).
    // Cavities are listed in order; a cavity without level-l tiles gets an
    // empty range.
    for (int l = 0; l < b->Lmax; ++l) {
        BatchRange &r = b->hr[1 + l];
        int sh = shape_of(b, l);
        r.count = C;
        int s = 0;
        for (int c = 0; c < C; ++c) {
            r.start[c] = s;
            int n = b->N[c] >> l;
            int gx = (n - 1 + tile_tx(sh) - 1) / tile_tx(sh), gy = (n - 1 + tile_ty(sh) - 1) / tile_ty(sh);
            r.gx[c] = gx;
            // shape 4: blocks of four warp tiles; otherwise one tile per block
            if (l < b->lc[c]) s += sh == 4 ? warp_tile_blocks(n) : gx * gy;
        }
        r.start[C] = s;
        b->rblocks[1 + l] = s;
    }
}

// Uploads the descriptors and ranges; once the batch runs, the cavities'
// device-side solve state (counters, logs, status) is kept.
int upload_tables(lc_batch *b) {
    cudaStream_t s = b->stream();
    if (b->initialized) {
        std::vector<BatchCav> cur(b->count);
        LB_CUDA(cudaMemcpyAsync(cur.data(), b->dcav(), sizeof(BatchCav) * b->count, cudaMemcpyDeviceToHost, s));
        LB_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < b->count; ++c) {
            BatchCav &h = b->hcav[c];
            h.active = cur[c].active;
            h.cycles = cur[c].cycles;
            h.status = cur[c].status;
            h.last_cycles = cur[c].last_cycles;
            h.arrive = cur[c].arrive;
            h.last_rel = cur[c].last_rel;
            h.nsolves = cur[c].nsolves;
        }
    }
    LB_CUDA(cudaMemcpyAsync(b->dcav(), b->hcav.data(), sizeof(BatchCav) * b->count, cudaMemcpyHostToDevice, s));
    LB_CUDA(cudaMemcpyAsync(b->drange(0), b->hr.data(), sizeof(BatchRange) * b->hr.size(), cudaMemcpyHostToDevice, s));
    LB_CUDA(cudaStreamSynchronize(s));
    return LC_OK;
}

void release_graph(lc_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->dirty = true;
}

// One cycle for every active cavity: FP32 V-cycle on the correction, psi64 +=
// e, FP64 residual, per-cavity stopping rule and the loop condition.
int enqueue_cycle(lc_batch *b, cudaStream_t s, cudaGraphConditionalHandle h) {
    float beta = (float)b->beta;
    for (int l = 0; l < b->Lmax; ++l)
        if (b->rblocks[1 + l])
            LB_CUDA(launch_down_batch<float>(s, shape_of(b, l), b->op, b->dcav(), b->drange(1 + l), l,
                                             b->rblocks[1 + l], b->nu1, beta));
    LB_CUDA(launch_coarse_batch(s, b->op, b->dcav(), b->count, (int)b->coarse_smem, b->nu1, b->nu2,
                                b->coarse_direct ? 0 : b->nuc, beta));
    for (int l = b->Lmax - 1; l >= 0; --l)
        if (b->rblocks[1 + l])
            LB_CUDA(launch_up_batch<float>(s, shape_of(b, l), b->op, b->dcav(), b->drange(1 + l), l,
                                           b->rblocks[1 + l], b->nu2, beta));
    BatchFinish fin{1, b->tol, b->max_cycles, h, b->dstate()};
    LB_CUDA(launch_residual_batch(s, b->op, b->dcav(), b->drange(kResRange), b->drange(0), b->rblocks[kResRange],
                                  b->at<double>(b->lay.rpart),
                                  b->at<double>(b->lay.gpart), fin));
    return LC_OK;
}

int enqueue_head(lc_batch *b, cudaStream_t s, int stage) {
    LB_CUDA(launch_stage_batch(s, b->dcav(), b->drange(0), b->rblocks[0], stage, b->advect, b->rhs64));
    LB_CUDA(launch_assemble_batch(s, b->op, b->dcav(), b->drange(0), b->rblocks[0], stage,
                                  b->at<double>(b->lay.gpart)));
    BatchFinish none{0, 0.0, 0, 0, nullptr};
    LB_CUDA(launch_residual_batch(s, b->op, b->dcav(), b->drange(kResRange), b->drange(0), b->rblocks[kResRange],
                                  b->at<double>(b->lay.rpart),
                                  b->at<double>(b->lay.gpart), none));
    return LC_OK;
}

int build_graph_once(lc_batch *b);

// Builds the step graph, without programmatic-dependent-launch edges if it
// cannot be built with them.
int build_graph(lc_batch *b) {
    int rc;
    {
        PdlScope pdl(b->pdl && !b->pdl_unsupported);
        rc = build_graph_once(b);
    }
    if (rc != LC_OK && b->pdl && !b->pdl_unsupported) {
        cudaGetLastError();  // clear a launch error of the failed capture
        b->pdl_unsupported = true;
        rc = build_graph_once(b);
    }
    return rc;
}

int build_graph_once(lc_batch *b) {
    release_graph(b);
    cudaStream_t s;
    LB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return bcuda(e, "cudaStreamBeginCapture");
    }
    int rc = LC_OK;
    for (int k = 0; k < 5 && rc == LC_OK; ++k) {
        rc = enqueue_head(b, s, k);
        if (rc) break;
        cudaStreamCaptureStatus cst;
        cudaGraph_t g;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd);
        cudaGraphConditionalHandle h = 0;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
        if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(b->cap2, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = bcuda(e, "conditional node");
            break;
        }
        rc = enqueue_cycle(b, b->cap2, h);
        cudaGraph_t tmp = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap2, &tmp);
        if (rc) break;
        if (e2 != cudaSuccess) {
            rc = bcuda(e2, "cudaStreamEndCapture(body)");
            break;
        }
        e = b->rhs64 ? cudaSuccess : launch_psi32_batch(s, b->dcav(), b->drange(0), b->rblocks[0]);
        if (e == cudaSuccess) e = launch_thom_batch(s, b->dcav(), b->count, b->U);
        if (e != cudaSuccess) rc = bcuda(e, "launch_thom_batch");
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    cudaStreamDestroy(s);
    if (rc != LC_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bcuda(e, "cudaStreamEndCapture");
    b->graph = g;
    LB_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->dirty = false;
    return LC_OK;
}

int eager_step(lc_batch *b) {
    static const char *kStageName[5] = {"stage 1", "stage 2", "stage 3", "stage 4", "stage 5"};
    PdlScope pdl(b->pdl);
    cudaStream_t s = b->stream();
    for (int k = 0; k < 5; ++k) {
        NvtxRange stage_range(kStageName[k]);
        int rc = enqueue_head(b, s, k);
        if (rc) return rc;
        for (;;) {
            NvtxRange cycle_range("poisson cycle");
            rc = enqueue_cycle(b, s, 0);
            if (rc) return rc;
            int more = 0;
            LB_CUDA(cudaMemcpyAsync(&more, &b->dstate()->more, sizeof(int), cudaMemcpyDeviceToHost, s));
            LB_CUDA(cudaStreamSynchronize(s));
            if (!more) break;
        }
        if (!b->rhs64) LB_CUDA(launch_psi32_batch(s, b->dcav(), b->drange(0), b->rblocks[0]));
        LB_CUDA(launch_thom_batch(s, b->dcav(), b->count, b->U));
    }
    return LC_OK;
}

int binit(lc_batch *b) {
    if (b->initialized) return LC_OK;
    LB_CUDA(init_mg_kernel_attributes());
    if (!b->ws) {
        void *p = nullptr;
        LB_CUDA(cudaMalloc(&p, b->lay.total));
        b->ws = static_cast<char *>(p);
        b->ws_bytes = b->lay.total;
        b->ws_owned = true;
    }
    if (!b->own) LB_CUDA(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
    if (!b->cap2) LB_CUDA(cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking));
    LB_CUDA(cudaMemsetAsync(b->ws, 0, b->lay.total, b->stream()));
    fill_tables(b);
    int rc = upload_tables(b);
    if (rc) return rc;
    LB_CUDA(launch_thom_batch(b->stream(), b->dcav(), b->count, b->U));
    b->initialized = true;
    return LC_OK;
}

// Reads each cavity's status after a sync; reports (and clears) the first error.
int bsync(lc_batch *b) {
    if (!b->initialized) return LC_OK;
    LB_CUDA(cudaStreamSynchronize(b->stream()));
    std::vector<BatchCav> v(b->count);
    LB_CUDA(cudaMemcpy(v.data(), b->dcav(), sizeof(BatchCav) * b->count, cudaMemcpyDeviceToHost));
    int err = LC_OK;
    for (int c = 0; c < b->count; ++c) {
        if (v[c].status) {
            int zero = 0;
            LB_CUDA(cudaMemcpy(&b->dcav()[c].status, &zero, sizeof(int), cudaMemcpyHostToDevice));
            if (err == LC_OK) {
                if (v[c].status & kStatusNonFinite)
                    err = bfail(LC_ERR_NONFINITE, "non-finite residual in cavity " + std::to_string(c));
                else
                    err = bfail(LC_ERR_NOCONV, "Poisson solve reached max_cycles in cavity " + std::to_string(c));
            }
        }
    }
    return err;
}

}  // namespace

extern "C" {

size_t lc_batch_workspace_bytes(int count, const int *N, int precision) {
    if (count < 1 || count > kMaxBatch || !N || precision != LC_PREC_MIXED) return 0;
    lc_batch tmp;
    tmp.count = count;
    tmp.N.assign(N, N + count);
    for (int c = 0; c < count; ++c)
        if (N[c] < 128 || N[c] > 8192 || nlevels(N[c]) < 2) return 0;
    return plan(&tmp) ? tmp.lay.total : 0;
}

lc_batch *lc_batch_create(int count, const int *N, const double *Re, const double *dt, double tol, int precision) {
    if (count < 1 || count > kMaxBatch || !N || !Re) {
        bfail(LC_ERR_ARG, "count must be 1..256 with N and Re arrays");
        return nullptr;
    }
    if (precision != LC_PREC_MIXED) {
        bfail(LC_ERR_ARG, "the batched engine runs the mixed-precision step (precision = LC_PREC_MIXED)");
        return nullptr;
    }
    if (!(tol > 0.0) || !std::isfinite(tol)) {
        bfail(LC_ERR_ARG, "tol must be positive");
        return nullptr;
    }
    lc_batch *b = new lc_batch();
    b->count = count;
    b->tol = tol;
    for (int c = 0; c < count; ++c) {
        if (N[c] < 128 || N[c] > 8192 || nlevels(N[c]) < 2 || !(Re[c] > 0.0) || !std::isfinite(Re[c])) {
            delete b;
            bfail(LC_ERR_ARG, "cavity " + std::to_string(c) + ": N must be 2^k, 3*2^k, 5*2^k or 7*2^k in 128..8192, Re > 0");
            return nullptr;
        }
        double h = 1.0 / N[c];
        double d = dt ? dt[c] : 0.0;
        if (!std::isfinite(d)) d = 0.0;
        if (d <= 0.0) d = 0.25 * std::fmin(h, Re[c] * h * h / 4.0);
        b->N.push_back(N[c]);
        b->Re.push_back(Re[c]);
        b->dt.push_back(d);
    }
    if (!plan(b)) {
        delete b;
        bfail(LC_ERR_ARG, "grid too small for the batched tile levels");
        return nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        g_blive.insert(b);
    }
    return b;
}

void lc_batch_destroy(lc_batch *b) {
    if (!blive(b)) return;
    {
        std::lock_guard<std::mutex> lk(g_bmu);
        g_blive.erase(b);
    }
    if (b->initialized) cudaStreamSynchronize(b->stream());
    release_graph(b);
    if (b->ws_owned && b->ws) cudaFree(b->ws);
    if (b->own) cudaStreamDestroy(b->own);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    delete b;
}

int lc_batch_set_option(lc_batch *b, const char *key, double v) {
    LB_CHECK(b);
    if (!key) return bfail(LC_ERR_ARG, "NULL option key");
    std::string k(key);
    int iv = (int)v;
    bool integral = v == (double)iv;
    if (k == "op" || k == "coarse_max" || k == "coarse_direct") {
        if (b->initialized) return bfail(LC_ERR_ARG, k + " must be set before first use");
        if (k == "op") {
            if (!integral || (iv != 0 && iv != 1)) return bfail(LC_ERR_ARG, "op must be 0 or 1");
            b->op = iv;
        } else if (k == "coarse_direct") {
            if (!integral || (iv != 0 && iv != 1)) return bfail(LC_ERR_ARG, "coarse_direct must be 0 or 1");
            b->coarse_direct = iv;
        } else {
            if (!integral || iv < 8 || iv > 64) return bfail(LC_ERR_ARG, "coarse_max must be 8..64");
            b->coarse_max = iv;
        }
        if (!plan(b)) return bfail(LC_ERR_ARG, "grid too small for the batched tile levels");
    } else if (k == "nu1" || k == "nu2") {
        if (!integral || iv < 1 || iv > 4) return bfail(LC_ERR_ARG, "nu1/nu2 must be 1..4");
        (k == "nu1" ? b->nu1 : b->nu2) = iv;
    } else if (k == "nuc") {
        if (!integral || iv < 1 || iv > 256) return bfail(LC_ERR_ARG, "nuc must be 1..256");
        b->nuc = iv;
    } else if (k == "beta") {
        if (!(v > 0.0 && v < 2.0)) return bfail(LC_ERR_ARG, "beta must be in (0, 2)");
        b->beta = v;
    } else if (k == "max_cycles") {
        if (!integral || iv < 1) return bfail(LC_ERR_ARG, "max_cycles must be >= 1");
        b->max_cycles = iv;
    } else if (k == "U") {
        if (!std::isfinite(v)) return bfail(LC_ERR_ARG, "U must be finite");
        b->U = v;
        if (b->initialized) LB_CUDA(launch_thom_batch(b->stream(), b->dcav(), b->count, b->U));
    } else if (k == "advect") {
        if (!integral || (iv != 0 && iv != 1)) return bfail(LC_ERR_ARG, "advect must be 0 or 1");
        b->advect = iv;
    } else if (k == "rhs64") {
        if (!integral || (iv != 0 && iv != 1)) return bfail(LC_ERR_ARG, "rhs64 must be 0 or 1");
        b->rhs64 = iv;
    } else if (k == "pdl") {
        if (!integral || (iv != 0 && iv != 1)) return bfail(LC_ERR_ARG, "pdl must be 0 or 1");
        b->pdl = iv;
        b->pdl_unsupported = false;
    } else if (k == "graph") {
        if (!integral || (iv != 0 && iv != 1)) return bfail(LC_ERR_ARG, "graph must be 0 or 1");
        b->use_graph = iv;
        return LC_OK;
    } else {
        return bfail(LC_ERR_ARG, "unknown option " + k);
    }
    if (b->initialized) {
        fill_tables(b);
        int rc = upload_tables(b);
        if (rc) return rc;
    }
    b->dirty = true;
    return LC_OK;
}

int lc_batch_set_stream(lc_batch *b, void *stream) {
    LB_CHECK(b);
    if (b->initialized) {
        cudaEvent_t ev;
        LB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        LB_CUDA(cudaEventRecord(ev, b->stream()));
        b->user = static_cast<cudaStream_t>(stream);
        b->use_user = true;
        LB_CUDA(cudaStreamWaitEvent(b->stream(), ev, 0));
        LB_CUDA(cudaEventDestroy(ev));
    } else {
        b->user = static_cast<cudaStream_t>(stream);
        b->use_user = true;
    }
    return LC_OK;
}

int lc_batch_bind_workspace(lc_batch *b, void *dev_ptr, size_t bytes) {
    LB_CHECK(b);
    if (b->initialized) return bfail(LC_ERR_ARG, "workspace must be bound before first use");
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255))
        return bfail(LC_ERR_SIZE, "workspace must be 256-byte aligned");
    if (bytes < b->lay.total) return bfail(LC_ERR_SIZE, "workspace smaller than lc_batch_workspace_bytes");
    b->ws = static_cast<char *>(dev_ptr);
    b->ws_bytes = bytes;
    b->ws_owned = false;
    return LC_OK;
}

int lc_batch_step(lc_batch *b, int nsteps) {
    LB_CHECK(b);
    if (nsteps < 0) return bfail(LC_ERR_ARG, "nsteps must be >= 0");
    NvtxRange range("lc_batch_step");
    int rc = binit(b);
    if (rc) return rc;
    if (b->use_graph && b->dirty) {
        rc = build_graph(b);
        if (rc) return rc;
    }
    for (int n = 0; n < nsteps; ++n) {
        if (b->use_graph) {
            LB_CUDA(cudaGraphLaunch(b->exec, b->stream()));
        } else {
            rc = eager_step(b);
            if (rc) return rc;
        }
        b->steps++;
    }
    return LC_OK;
}

int lc_batch_synchronize(lc_batch *b) {
    LB_CHECK(b);
    return bsync(b);
}

int lc_batch_get(lc_batch *b, int cavity, int field, double *host_out, size_t n_elems) {
    LB_CHECK(b);
    if (cavity < 0 || cavity >= b->count || field < 0 || field > 1 || !host_out)
        return bfail(LC_ERR_ARG, "bad cavity, field or buffer");
    int N = b->N[cavity];
    if (n_elems < (size_t)(N + 1) * (N + 1)) return bfail(LC_ERR_SIZE, "host buffer smaller than (N+1)^2");
    int rc = binit(b);
    if (rc) return rc;
    size_t off = field == 0 ? b->lay.psi64[cavity] : b->lay.W[0][cavity];
    LB_CUDA(cudaMemcpy2DAsync(host_out, (N + 1) * sizeof(double), b->at<double>(off), pitch32(N) * sizeof(double),
                              (N + 1) * sizeof(double), N + 1, cudaMemcpyDeviceToHost, b->stream()));
    return bsync(b);
}

int lc_batch_set_state(lc_batch *b, int cavity, const double *psi, const double *omega) {
    LB_CHECK(b);
    if (cavity < 0 || cavity >= b->count || !psi || !omega) return bfail(LC_ERR_ARG, "bad cavity or state arrays");
    int rc = binit(b);
    if (rc) return rc;
    int N = b->N[cavity], P = pitch32(N);
    cudaStream_t s = b->stream();
    size_t hp = (N + 1) * sizeof(double), dp = P * sizeof(double);
    double *d_psi = b->at<double>(b->lay.psi64[cavity]), *d_w = b->at<double>(b->lay.W[0][cavity]);
    LB_CUDA(cudaMemcpy2DAsync(d_psi, dp, psi, hp, hp, N + 1, cudaMemcpyHostToDevice, s));
    LB_CUDA(launch_zero_walls(s, d_psi, N, P));
    LB_CUDA(cudaMemcpy2DAsync(d_w, dp, omega, hp, hp, N + 1, cudaMemcpyHostToDevice, s));
    LB_CUDA(launch_to32(s, d_psi, P, b->at<float>(b->lay.psi32[cavity]), P, N));
    LB_CUDA(launch_to32(s, d_w, P, b->at<float>(b->lay.Ws[0][cavity]), P, N));
    LB_CUDA(launch_thom_batch(s, b->dcav(), b->count, b->U));
    LB_CUDA(cudaStreamSynchronize(s));
    return LC_OK;
}

int lc_batch_cycle_log(lc_batch *b, int cavity, int *out, size_t max, size_t *n_out) {
    LB_CHECK(b);
    if (cavity < 0 || cavity >= b->count || !out || !n_out) return bfail(LC_ERR_ARG, "bad cavity or output");
    int rc = binit(b);
    if (rc) return rc;
    rc = bsync(b);
    BatchCav v;
    LB_CUDA(cudaMemcpy(&v, b->dcav() + cavity, sizeof(BatchCav), cudaMemcpyDeviceToHost));
    std::vector<int> ring(kLogN);
    LB_CUDA(cudaMemcpy(ring.data(), v.log, sizeof(int) * kLogN, cudaMemcpyDeviceToHost));
    unsigned long long total = v.nsolves, avail = total < (unsigned long long)kLogN ? total : kLogN;
    size_t n = avail < max ? (size_t)avail : max;
    for (size_t k = 0; k < n; ++k) out[k] = ring[(total - avail + k) % kLogN];
    *n_out = n;
    return rc;
}

int lc_batch_info(lc_batch *b, int cavity, double out[8]) {
    LB_CHECK(b);
    if (cavity < 0 || cavity >= b->count || !out) return bfail(LC_ERR_ARG, "bad cavity or output");
    out[0] = b->N[cavity];
    out[1] = b->Re[cavity];
    out[2] = b->dt[cavity];
    out[3] = b->nv[cavity];
    out[4] = b->lc[cavity];
    out[5] = (double)b->steps;
    out[6] = b->Lmax > 0 ? shape_of(b, 0) : -1;
    out[7] = (double)b->lay.total;
    return LC_OK;
}

int lc_batch_autotune(lc_batch *b, int reps, int *shapes_out, int max_levels) {
    LB_CHECK(b);
    if (reps < 1 || !shapes_out || max_levels < 1) return bfail(LC_ERR_ARG, "bad reps or output");
    int rc = binit(b);
    if (rc) return rc;
    cudaStream_t s = b->stream();
    // the level-0 up kernel adds its correction to psi64: keep psi64 / psi32 and restore them
    std::vector<std::pair<size_t, size_t>> keep;
    size_t extra = 0;
    for (int c = 0; c < b->count; ++c) {
        size_t n0 = (size_t)(b->N[c] + 1) * pitch32(b->N[c]);
        keep.push_back({b->lay.psi64[c], n0 * 8});
        keep.push_back({b->lay.psi32[c], n0 * 4});
        extra += n0 * 12;
    }
    void *save = nullptr;
    LB_CUDA(cudaMalloc(&save, extra));
    size_t o = 0;
    for (auto &kv : keep) {
        LB_CUDA(cudaMemcpyAsync((char *)save + o, b->ws + kv.first, kv.second, cudaMemcpyDeviceToDevice, s));
        o += kv.second;
    }
    cudaEvent_t e0, e1;
    LB_CUDA(cudaEventCreate(&e0));
    LB_CUDA(cudaEventCreate(&e1));
    int nu = b->nu1 > b->nu2 ? b->nu1 : b->nu2;
    for (int l = 0; l < b->Lmax; ++l) {
        float best = 1e30f;
        int pick = -1;
        for (int sh = 0; sh < 5; ++sh) {
            if (tile_smem_bytes(sh, b->op, nu, 4) > kMaxSmem - 1024) continue;
            b->shape[l] = sh;
            fill_tables(b);
            rc = upload_tables(b);
            if (rc) break;
            auto run = [&]() -> cudaError_t {
                cudaError_t e = launch_down_batch<float>(s, sh, b->op, b->dcav(), b->drange(1 + l), l, b->rblocks[1 + l],
                                                         b->nu1, (float)b->beta);
                if (e == cudaSuccess)
                    e = launch_up_batch<float>(s, sh, b->op, b->dcav(), b->drange(1 + l), l, b->rblocks[1 + l],
                                               b->nu2, (float)b->beta);
                return e;
            };
            LB_CUDA(run());
            LB_CUDA(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r) LB_CUDA(run());
            LB_CUDA(cudaEventRecord(e1, s));
            LB_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            LB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                pick = sh;
            }
        }
        if (rc) break;
        b->shape[l] = pick;
        if (l < max_levels) shapes_out[l] = pick;
    }
    o = 0;
    for (auto &kv : keep) {
        LB_CUDA(cudaMemcpyAsync(b->ws + kv.first, (char *)save + o, kv.second, cudaMemcpyDeviceToDevice, s));
        o += kv.second;
    }
    LB_CUDA(cudaStreamSynchronize(s));
    cudaFree(save);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    fill_tables(b);
    rc = upload_tables(b);
    b->dirty = true;
    for (int l = b->Lmax; l < max_levels; ++l) shapes_out[l] = -1;
    return rc;
}

int lc_batch_autotune_schedule(lc_batch *b, int steps, int nu_out[2]) {
    LB_CHECK(b);
    if (steps < 1 || !nu_out) return bfail(LC_ERR_ARG, "bad steps or output");
    int rc = binit(b);
    if (rc) return rc;
    rc = bsync(b);  // report (and clear) an error from earlier work before timing
    if (rc) return rc;
    cudaStream_t s = b->stream();
    void *save = nullptr;
    LB_CUDA(cudaMalloc(&save, b->lay.total));
    LB_CUDA(cudaMemcpyAsync(save, b->ws, b->lay.total, cudaMemcpyDeviceToDevice, s));
    long long steps0 = b->steps;
    std::vector<int> shape0 = b->shape;
    int nu1_0 = b->nu1, nu2_0 = b->nu2;
    static const int kCand[6][2] = {{1, 1}, {2, 1}, {1, 2}, {2, 2}, {3, 1}, {3, 2}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    int pick = -1;
    rc = LC_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = bfail(LC_ERR_CUDA, "cudaEventCreate failed");
    for (int k = 0; k < 6 && rc == LC_OK; ++k) {
        b->nu1 = kCand[k][0];
        b->nu2 = kCand[k][1];
        b->shape.assign(b->Lmax, -1);
        fill_tables(b);
        rc = upload_tables(b);
        if (rc) break;
        b->dirty = true;
        rc = lc_batch_step(b, 1);
        if (rc) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = bfail(LC_ERR_CUDA, "cudaEventRecord failed");
        if (rc == LC_OK) rc = lc_batch_step(b, steps);
        if (rc == LC_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = bfail(LC_ERR_CUDA, "cudaEventRecord failed");
        if (rc) break;
        int st = bsync(b);  // a schedule whose solves hit max_cycles is not a candidate
        if (st == LC_ERR_CUDA) {
            rc = st;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = bfail(LC_ERR_CUDA, "cudaEventElapsedTime failed");
            break;
        }
        if (st == LC_OK && ms < best) {
            best = ms;
            pick = k;
        }
        // back to the state the tuner started from
        if (cudaMemcpyAsync(b->ws, save, b->lay.total, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            rc = bfail(LC_ERR_CUDA, "restoring the workspace failed");
        b->steps = steps0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaMemcpyAsync(b->ws, save, b->lay.total, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaFree(save);
    b->steps = steps0;
    if (rc == LC_OK && pick < 0) rc = bfail(LC_ERR_NOCONV, "no smoothing schedule converged");
    if (rc == LC_OK) {
        b->nu1 = kCand[pick][0];
        b->nu2 = kCand[pick][1];
        b->shape.assign(b->Lmax, -1);
        nu_out[0] = b->nu1;
        nu_out[1] = b->nu2;
    } else {
        b->nu1 = nu1_0;
        b->nu2 = nu2_0;
        b->shape = shape0;
    }
    fill_tables(b);
    int rc2 = upload_tables(b);
    b->dirty = true;
    return rc ? rc : rc2;
}

}  // extern "C"
