// Batched sweeps: many independent cases advanced together (include/lbm.h,
// "batched sweeps").  Host side: validation, the batch arrays, size classes
// and their work lists, the CUDA graphs of the step and the autotuner.
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.cuh"

extern template struct lbm::Launch<lbm::D2Q9, lbm::StoreF32>;
extern template struct lbm::Launch<lbm::D2Q9, lbm::StoreF16>;
extern template struct lbm::Launch<lbm::D3Q19, lbm::StoreF32>;
extern template struct lbm::Launch<lbm::D3Q19, lbm::StoreF16>;
extern template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF32, 32, 1>;
extern template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF32, 64, 1>;
extern template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF32, 128, 1>;
extern template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF16, 32, 1>;
extern template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF16, 64, 1>;
extern template struct lbm::BatchLaunch<lbm::D2Q9, lbm::StoreF16, 128, 1>;
extern template struct lbm::BatchLaunch<lbm::D3Q19, lbm::StoreF32, 32, 8>;
extern template struct lbm::BatchLaunch<lbm::D3Q19, lbm::StoreF16, 32, 8>;

namespace lbm {
int api_validate(const lbm_params* p, std::string& why);
DevParams api_make_dev(const lbm_params* p, int64_t N);
void api_fill_diag(const DiagPartial& r, lbm_diag_out* out);
}  // namespace lbm

using lbm::BatchCase;
using lbm::BatchLaunch;
using lbm::D2Q9;
using lbm::D3Q19;
using lbm::DevParams;
using lbm::DiagPartial;
using lbm::FusedGeom;
using lbm::Launch;
using lbm::StoreF16;
using lbm::StoreF32;

namespace {

constexpr int kGraphSteps = 16;            // steps per graph replay (even: A/B parity is kept)
constexpr int kDiagParts = 2 * 152;
constexpr int64_t kCaseAlignNodes = 128;   // case planes start 256-byte aligned at 2-byte storage
const int kClassNxMax[] = {96, 192, 384, INT_MAX};

// Calls fn with a default-constructed Launch<lattice, storage>.
template <class Fn>
cudaError_t with_launch(int D, int storage, Fn fn)
{
    if (D == 2) return storage == 1 ? fn(Launch<D2Q9, StoreF16>{}) : fn(Launch<D2Q9, StoreF32>{});
    return storage == 1 ? fn(Launch<D3Q19, StoreF16>{}) : fn(Launch<D3Q19, StoreF32>{});
}

// Calls fn with a default-constructed BatchLaunch of the tile width tx.
template <class Fn>
cudaError_t with_batch(int D, int storage, int tx, Fn fn)
{
    if (D == 3) return storage == 1 ? fn(BatchLaunch<D3Q19, StoreF16, 32, 8>{}) : fn(BatchLaunch<D3Q19, StoreF32, 32, 8>{});
    if (storage == 1) {
        if (tx == 32) return fn(BatchLaunch<D2Q9, StoreF16, 32, 1>{});
        if (tx == 64) return fn(BatchLaunch<D2Q9, StoreF16, 64, 1>{});
        return fn(BatchLaunch<D2Q9, StoreF16, 128, 1>{});
    }
    if (tx == 32) return fn(BatchLaunch<D2Q9, StoreF32, 32, 1>{});
    if (tx == 64) return fn(BatchLaunch<D2Q9, StoreF32, 64, 1>{});
    return fn(BatchLaunch<D2Q9, StoreF32, 128, 1>{});
}

bool valid_tile(int D, int tx) { return D == 3 ? tx == 32 : (tx == 32 || tx == 64 || tx == 128); }

thread_local std::string g_batch_create_err;

}  // namespace

struct lbm_batch {
    int D = 2, Q = 9, storage = 0;
    size_t elem = 4;
    int ncases = 0;
    std::vector<lbm_params> params;
    std::vector<DevParams> dp;
    std::vector<int64_t> node_off;         // first (padded) node of each case in the batch
    std::vector<char> initialised;
    int64_t total_nodes = 0, max_nodes = 0;
    void *fA = nullptr, *gA = nullptr, *fB = nullptr, *gB = nullptr;   // A = current state
    float* phi = nullptr;                  // scratch of the largest case
    float* fref = nullptr;                 // float16 storage: f references of every case's planes
    DiagPartial* part = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, sms = 0;

    struct Class {
        std::vector<int> cases;            // batch indices of the class's cases
        int tx = 128, seglen = 32, bps = 1, occ = 1;
        BatchCase* d_cases = nullptr;
        int2* d_items = nullptr;
        int nitems = 0, cap_items = 0;
        cudaStream_t s = nullptr;
        cudaEvent_t done = nullptr;
        double ms = 0.0;
    };
    std::vector<Class> cls;
    int nx_max[LBM_BATCH_MAX_CLASSES] = {};
    int* counters = nullptr;               // one work counter per class
    cudaEvent_t fork = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // by the A/B parity at the start
    int parity = 0;
    std::string err;
};

static int bfail(lbm_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_batch_create_err = msg;
    return code;
}

static int bcuda(lbm_batch* b, cudaError_t e, const char* where)
{
    return bfail(b, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
                 std::string(where) + ": " + cudaGetErrorString(e));
}

#define BATCH_CUDA(b, call)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call); \
    } while (0)

static void drop_graphs(lbm_batch* b)
{
    for (cudaGraphExec_t& g : b->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Work list and case table of class k for its tile width and segment length.
static int build_class(lbm_batch* b, int k)
{
    lbm_batch::Class& c = b->cls[k];
    const int TY = b->D == 3 ? 8 : 1;
    std::vector<BatchCase> tab(c.cases.size());
    std::vector<int2> items;
    for (size_t i = 0; i < c.cases.size(); ++i) {
        const int ci = c.cases[i];
        const lbm_params& p = b->params[ci];
        BatchCase& bc = tab[i];
        std::memset(&bc, 0, sizeof bc);
        bc.P = b->dp[ci];
        bc.off = b->node_off[ci] * b->Q;
        const int nm = b->D == 3 ? p.nz : p.ny;
        FusedGeom& G = bc.G;
        G.tiles_x = (p.nx + c.tx - 1) / c.tx;
        G.tiles_y = b->D == 3 ? (p.ny + TY - 1) / TY : 1;
        G.ntiles = G.tiles_x * G.tiles_y;
        G.seglen = std::min(c.seglen, nm);
        G.nseg = (nm + G.seglen - 1) / G.seglen;
        G.items = G.ntiles * G.nseg;
        for (int it = 0; it < G.items; ++it) items.push_back(make_int2(int(i), it));
    }
    if (int(items.size()) > c.cap_items) {
        cudaFree(c.d_items);
        c.d_items = nullptr;
        BATCH_CUDA(b, cudaMalloc(reinterpret_cast<void**>(&c.d_items), items.size() * sizeof(int2)));
        c.cap_items = int(items.size());
    }
    if (!c.d_cases) BATCH_CUDA(b, cudaMalloc(reinterpret_cast<void**>(&c.d_cases), tab.size() * sizeof(BatchCase)));
    BATCH_CUDA(b, cudaMemcpyAsync(c.d_cases, tab.data(), tab.size() * sizeof(BatchCase), cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaMemcpyAsync(c.d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    c.nitems = int(items.size());
    int occ = 1;
    BATCH_CUDA(b, with_batch(b->D, b->storage, c.tx, [&](auto l) { return decltype(l)::setup(&occ); }));
    c.occ = std::max(occ, 1);
    c.bps = std::min(std::max(c.bps, 1), c.occ);
    drop_graphs(b);
    return LBM_OK;
}

// One step of class k from (fA, gA) into (fB, gB) on stream s.
static cudaError_t launch_class(lbm_batch* b, int k, cudaStream_t s, const void* fA, const void* gA, void* fB, void* gB)
{
    lbm_batch::Class& c = b->cls[k];
    const int nblocks = std::max(1, std::min(c.nitems, b->sms * c.bps));
    return with_batch(b->D, b->storage, c.tx, [&](auto l) {
        return decltype(l)::step(c.d_cases, c.d_items, c.nitems, b->counters + k, nblocks, fA, gA, fB, gB, s);
    });
}

// One step of the batch: the classes run on their own streams, forked from
// and joined back into the batch stream; then A and B swap.
static cudaError_t enqueue_step(lbm_batch* b)
{
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (size_t k = 0; k < b->cls.size() && e == cudaSuccess; ++k) {
        lbm_batch::Class& c = b->cls[k];
        e = cudaStreamWaitEvent(c.s, b->fork, 0);
        if (e == cudaSuccess) e = launch_class(b, int(k), c.s, b->fA, b->gA, b->fB, b->gB);
        if (e == cudaSuccess) e = cudaEventRecord(c.done, c.s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, c.done, 0);
    }
    std::swap(b->fA, b->fB);
    std::swap(b->gA, b->gB);
    b->parity ^= 1;
    return e;
}

static int capture_graph(lbm_batch* b)
{
    const int p = b->parity;
    cudaGraph_t g = nullptr;
    BATCH_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) e = enqueue_step(b);
    // an even number of swaps: the pointers and the parity are as before
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[p], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph[p] = nullptr;
        return bcuda(b, e, "batch step graph");
    }
    return LBM_OK;
}

static lbm::Buffers case_buffers(const lbm_batch* b, int c)
{
    const size_t off = size_t(b->node_off[c]) * b->Q * b->elem;
    lbm::Buffers bu;
    bu.fA = static_cast<char*>(b->fA) + off;
    bu.gA = static_cast<char*>(b->gA) + off;
    bu.fB = static_cast<char*>(b->fB) + off;
    bu.gB = static_cast<char*>(b->gB) + off;
    bu.phi = b->phi;
    bu.inplace = 0;
    bu.par = 0;
    return bu;
}

extern "C" {

int lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return LBM_OK;
    if (b->stream || b->own_stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (lbm_batch::Class& c : b->cls) {
        if (c.s) cudaStreamSynchronize(c.s);
        cudaFree(c.d_cases);
        cudaFree(c.d_items);
        if (c.done) cudaEventDestroy(c.done);
        if (c.s) cudaStreamDestroy(c.s);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->fA); cudaFree(b->gA); cudaFree(b->fB); cudaFree(b->gB);
    cudaFree(b->phi); cudaFree(b->part); cudaFree(b->counters); cudaFree(b->fref);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

int lbm_batch_create(const lbm_params* params, int32_t ncases, void* stream, lbm_batch** out)
{
    if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!params || ncases < 1) return bfail(nullptr, LBM_ERR_ARG, "need params and ncases >= 1");
    for (int c = 0; c < ncases; ++c) {
        const lbm_params* p = params + c;
        std::string why;
        if (lbm::api_validate(p, why) != 0) return bfail(nullptr, LBM_ERR_ARG, "case " + std::to_string(c) + ": " + why);
        if (p->lattice != params[0].lattice || p->storage != params[0].storage)
            return bfail(nullptr, LBM_ERR_ARG, "case " + std::to_string(c) + ": lattice and storage must match case 0");
        if (p->storage > 1) return bfail(nullptr, LBM_ERR_ARG, "batches store float32 or float16 (storage 0 or 1)");
        if (p->layout != 0) return bfail(nullptr, LBM_ERR_ARG, "batches use the A/B layout (layout 0)");
        for (int f = 0; f < 6; ++f)
            if (p->bc[f] != LBM_BC_PERIODIC && p->bc[f] != LBM_BC_WALL)
                return bfail(nullptr, LBM_ERR_ARG, "case " + std::to_string(c) + ": batch faces are periodic or wall");
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return bfail(nullptr, LBM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));

    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ERR_OOM, "host allocation failed");
    auto give_up = [&](int r) {
        g_batch_create_err = b->err;
        lbm_batch_destroy(b);
        return r;
    };
    b->D = params[0].lattice == LBM_D2Q9 ? 2 : 3;
    b->Q = b->D == 2 ? 9 : 19;
    b->storage = params[0].storage;
    b->elem = b->storage == 0 ? 4 : 2;
    b->ncases = ncases;
    b->params.assign(params, params + ncases);
    b->initialised.assign(ncases, 0);
    for (int c = 0; c < ncases; ++c) {
        const int64_t n = int64_t(params[c].nx) * params[c].ny * params[c].nz;
        // every case's planes start on a 128-node boundary: with 2-byte storage
        // an odd node count would otherwise leave the next case (and the
        // float32 fields staged in its B planes) 2-byte aligned
        b->total_nodes = (b->total_nodes + kCaseAlignNodes - 1) / kCaseAlignNodes * kCaseAlignNodes;
        b->node_off.push_back(b->total_nodes);
        if ((b->total_nodes * b->Q * int64_t(b->elem)) % 256 != 0)
            return give_up(bfail(b, LBM_ERR_ARG, "internal: case offset not 256-byte aligned"));
        b->dp.push_back(lbm::api_make_dev(params + c, n));
        b->total_nodes += b->dp.back().Np;        // blocked layout: rows padded to 32 nodes
        b->max_nodes = std::max(b->max_nodes, n);
    }
    cudaGetDevice(&b->device);
    if ((e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device)) != cudaSuccess)
        return give_up(bcuda(b, e, "device attributes"));
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if ((e = cudaStreamCreate(&b->stream)) != cudaSuccess) return give_up(bcuda(b, e, "stream"));
        b->own_stream = true;
    }
    const size_t bytes = size_t(b->total_nodes) * b->Q * b->elem;
    void** bufs[4] = {&b->fA, &b->gA, &b->fB, &b->gB};
    for (void** p : bufs)
        if ((e = cudaMalloc(p, bytes)) != cudaSuccess) return give_up(bcuda(b, e, "cudaMalloc(populations)"));
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->phi), size_t(b->max_nodes) * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&b->part), (kDiagParts + 1) * sizeof(DiagPartial))) != cudaSuccess)
        return give_up(bcuda(b, e, "cudaMalloc"));
    if (b->storage == 1) {
        // one reference per plane of the march axis per case, zero until the
        // case is initialised
        size_t nref = 0;
        for (int c = 0; c < ncases; ++c) nref += size_t(b->D == 2 ? params[c].ny : params[c].nz);
        if ((e = cudaMalloc(reinterpret_cast<void**>(&b->fref), nref * sizeof(float))) != cudaSuccess ||
            (e = cudaMemset(b->fref, 0, nref * sizeof(float))) != cudaSuccess)
            return give_up(bcuda(b, e, "cudaMalloc(references)"));
        for (int c = 0, o = 0; c < ncases; ++c) {
            b->dp[c].fref = b->fref + o;
            o += b->D == 2 ? params[c].ny : params[c].nz;
        }
    }
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess)
        return give_up(bcuda(b, e, "event"));

    // size classes by nx; empty ones are dropped
    const int nclass_all = int(sizeof(kClassNxMax) / sizeof(int));
    for (int k = 0, lo = 0; k < nclass_all; lo = kClassNxMax[k], ++k) {
        lbm_batch::Class c;
        for (int i = 0; i < ncases; ++i)
            if (params[i].nx > lo && params[i].nx <= kClassNxMax[k]) c.cases.push_back(i);
        if (c.cases.empty()) continue;
        b->nx_max[b->cls.size()] = kClassNxMax[k];
        c.tx = b->D == 3 ? 32 : (kClassNxMax[k] <= 96 ? 64 : 128);
        c.seglen = b->D == 3 ? 16 : 32;
        c.bps = INT_MAX;                   // clamped to the occupancy by build_class
        b->cls.push_back(c);
    }
    if ((e = cudaMalloc(reinterpret_cast<void**>(&b->counters), b->cls.size() * sizeof(int))) != cudaSuccess)
        return give_up(bcuda(b, e, "cudaMalloc(counters)"));
    for (size_t k = 0; k < b->cls.size(); ++k) {
        lbm_batch::Class& c = b->cls[k];
        if ((e = cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming)) != cudaSuccess)
            return give_up(bcuda(b, e, "class stream"));
        const int r = build_class(b, int(k));
        if (r != LBM_OK) return give_up(r);
    }
    *out = b;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b)
{
    return b ? b->err.c_str() : g_batch_create_err.c_str();
}

int lbm_batch_sync(lbm_batch* b)
{
    if (!b) return LBM_ERR_ARG;
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_init_fields(lbm_batch* b, int32_t c, const float* phi, const float* u, const float* pstar,
                          int32_t on_device)
{
    if (!b) return LBM_ERR_ARG;
    if (c < 0 || c >= b->ncases) return bfail(b, LBM_ERR_ARG, "case index out of range");
    if (!phi) return bfail(b, LBM_ERR_ARG, "phi is NULL");
    const int64_t N = b->dp[c].N;
    const lbm::Buffers bu = case_buffers(b, c);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t nb = size_t(N) * sizeof(float);
    // stage the fields in the case's f planes of B (Q * elem >= 4 (D + 2) bytes per node)
    float* s_phi = static_cast<float*>(bu.fB);
    float* s_u = s_phi + N;
    float* s_p = s_phi + N * (1 + b->D);
    BATCH_CUDA(b, cudaMemcpyAsync(s_phi, phi, nb, kind, b->stream));
    if (u) BATCH_CUDA(b, cudaMemcpyAsync(s_u, u, nb * b->D, kind, b->stream));
    if (pstar) BATCH_CUDA(b, cudaMemcpyAsync(s_p, pstar, nb, kind, b->stream));
    cudaError_t e = with_launch(b->D, b->storage, [&](auto l) {
        const float* vp = pstar ? s_p : nullptr;
        cudaError_t r = b->fref ? decltype(l)::plane_ref(b->dp[c], vp, 1.0f, const_cast<float*>(b->dp[c].fref),
                                                         b->stream)
                                : cudaSuccess;
        if (r == cudaSuccess) r = decltype(l)::init(b->dp[c], s_phi, u ? s_u : nullptr, vp, bu.fA, bu.gA, b->stream);
        return r;
    });
    if (e != cudaSuccess) return bcuda(b, e, "init kernel");
    if (!on_device) BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    b->initialised[c] = 1;
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps)
{
    if (!b) return LBM_ERR_ARG;
    if (nsteps < 0) return bfail(b, LBM_ERR_ARG, "nsteps < 0");
    for (int c = 0; c < b->ncases; ++c)
        if (!b->initialised[c]) return bfail(b, LBM_ERR_STATE, "case " + std::to_string(c) + " is not initialised");
    while (nsteps >= kGraphSteps) {
        if (!b->graph[b->parity]) {
            const int r = capture_graph(b);
            if (r != LBM_OK) return r;
        }
        BATCH_CUDA(b, cudaGraphLaunch(b->graph[b->parity], b->stream));
        nsteps -= kGraphSteps;
    }
    for (; nsteps > 0; --nsteps) {
        cudaError_t e = enqueue_step(b);
        if (e != cudaSuccess) return bcuda(b, e, "batch step");
    }
    return LBM_OK;
}

int lbm_batch_get_fields(lbm_batch* b, int32_t c, float* phi, float* u, float* p, int32_t on_device)
{
    if (!b) return LBM_ERR_ARG;
    if (c < 0 || c >= b->ncases) return bfail(b, LBM_ERR_ARG, "case index out of range");
    if (!b->initialised[c]) return bfail(b, LBM_ERR_STATE, "case is not initialised");
    const int64_t N = b->dp[c].N;
    const lbm::Buffers bu = case_buffers(b, c);
    float* o_phi = static_cast<float*>(bu.fB);
    float* o_u = o_phi + N;
    float* o_p = o_phi + N * (1 + b->D);
    cudaError_t e = with_launch(b->D, b->storage,
                                [&](auto l) { return decltype(l)::fields(b->dp[c], bu, o_phi, o_u, o_p, b->stream); });
    if (e != cudaSuccess) return bcuda(b, e, "fields kernel");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t nb = size_t(N) * sizeof(float);
    if (phi) BATCH_CUDA(b, cudaMemcpyAsync(phi, o_phi, nb, kind, b->stream));
    if (u) BATCH_CUDA(b, cudaMemcpyAsync(u, o_u, nb * b->D, kind, b->stream));
    if (p) BATCH_CUDA(b, cudaMemcpyAsync(p, o_p, nb, kind, b->stream));
    if (!on_device) BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

int lbm_batch_diag(lbm_batch* b, int32_t c, double phase_eps, lbm_diag_out* out)
{
    if (!b || !out) return LBM_ERR_ARG;
    if (c < 0 || c >= b->ncases) return bfail(b, LBM_ERR_ARG, "case index out of range");
    if (!b->initialised[c]) return bfail(b, LBM_ERR_STATE, "case is not initialised");
    const lbm::Buffers bu = case_buffers(b, c);
    cudaError_t e = with_launch(b->D, b->storage, [&](auto l) {
        return decltype(l)::diag(b->dp[c], bu, phase_eps, b->part, kDiagParts, b->part + kDiagParts, b->stream);
    });
    if (e != cudaSuccess) return bcuda(b, e, "diag kernels");
    DiagPartial r;
    BATCH_CUDA(b, cudaMemcpyAsync(&r, b->part + kDiagParts, sizeof r, cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    lbm::api_fill_diag(r, out);
    if (r.nonfinite) return bfail(b, LBM_ERR_DIVERGED, "non-finite populations");
    return LBM_OK;
}

int lbm_batch_get_plan(const lbm_batch* b, lbm_batch_plan* plan)
{
    if (!b || !plan) return LBM_ERR_ARG;
    std::memset(plan, 0, sizeof *plan);
    plan->nclasses = int32_t(b->cls.size());
    for (size_t k = 0; k < b->cls.size(); ++k) {
        const lbm_batch::Class& c = b->cls[k];
        plan->nx_max[k] = b->nx_max[k];
        plan->ncases[k] = int32_t(c.cases.size());
        plan->tile_x[k] = c.tx;
        plan->seglen[k] = c.seglen;
        plan->blocks_per_sm[k] = c.bps;
        plan->ms_per_step[k] = c.ms;
    }
    return LBM_OK;
}

int lbm_batch_set_plan(lbm_batch* b, const lbm_batch_plan* plan)
{
    if (!b || !plan) return LBM_ERR_ARG;
    if (plan->nclasses != int32_t(b->cls.size())) return bfail(b, LBM_ERR_ARG, "plan: class count differs");
    for (size_t k = 0; k < b->cls.size(); ++k) {
        if (plan->nx_max[k] != b->nx_max[k] || plan->ncases[k] != int32_t(b->cls[k].cases.size()))
            return bfail(b, LBM_ERR_ARG, "plan: classes differ from the batch's");
        if (!valid_tile(b->D, plan->tile_x[k])) return bfail(b, LBM_ERR_ARG, "plan: tile_x not available");
        if (plan->seglen[k] < 1 || plan->blocks_per_sm[k] < 1) return bfail(b, LBM_ERR_ARG, "plan: seglen and blocks_per_sm must be >= 1");
    }
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k < b->cls.size(); ++k) {
        lbm_batch::Class& c = b->cls[k];
        c.tx = plan->tile_x[k];
        c.seglen = plan->seglen[k];
        c.bps = plan->blocks_per_sm[k];
        const int r = build_class(b, int(k));
        if (r != LBM_OK) return r;
        if (plan->blocks_per_sm[k] > c.occ) return bfail(b, LBM_ERR_ARG, "plan: blocks_per_sm above the occupancy");
    }
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int32_t trial_steps, lbm_batch_plan* plan)
{
    if (!b) return LBM_ERR_ARG;
    if (trial_steps < 1) return bfail(b, LBM_ERR_ARG, "trial_steps must be >= 1");
    for (int c = 0; c < b->ncases; ++c)
        if (!b->initialised[c]) return bfail(b, LBM_ERR_STATE, "tune needs every case initialised");
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    cudaEvent_t t0, t1;
    BATCH_CUDA(b, cudaEventCreate(&t0));
    cudaError_t e = cudaEventCreate(&t1);
    if (e != cudaSuccess) {
        cudaEventDestroy(t0);
        return bcuda(b, e, "cudaEventCreate");
    }
    int rc = LBM_OK;
    for (size_t k = 0; k < b->cls.size() && rc == LBM_OK; ++k) {
        lbm_batch::Class& c = b->cls[k];
        std::vector<int> txs = b->D == 3 ? std::vector<int>{32} : std::vector<int>{32, 64, 128};
        std::vector<int> segs = b->D == 3 ? std::vector<int>{4, 8, 16, 32} : std::vector<int>{4, 16, 64};
        double best = 1e300;
        int btx = c.tx, bseg = c.seglen, bbps = c.bps;
        for (int tx : txs) {
            for (int seg : segs) {
                c.tx = tx;
                c.seglen = seg;
                c.bps = INT_MAX;
                if ((rc = build_class(b, int(k))) != LBM_OK) break;
                const int occ = c.occ;
                for (int bps : {occ, std::max(1, occ / 2)}) {
                    c.bps = bps;
                    // one step from the current state, repeated: A is only read
                    e = launch_class(b, int(k), b->stream, b->fA, b->gA, b->fB, b->gB);
                    if (e == cudaSuccess) e = cudaEventRecord(t0, b->stream);
                    for (int s = 0; s < trial_steps && e == cudaSuccess; ++s)
                        e = launch_class(b, int(k), b->stream, b->fA, b->gA, b->fB, b->gB);
                    if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                    if (e != cudaSuccess) {
                        rc = bcuda(b, e, "tuning launch");
                        break;
                    }
                    const double per = double(ms) / trial_steps;
                    if (per < best) {
                        best = per;
                        btx = tx;
                        bseg = seg;
                        bbps = bps;
                    }
                    if (occ == 1) break;
                }
                if (rc != LBM_OK) break;
            }
            if (rc != LBM_OK) break;
        }
        if (rc != LBM_OK) break;
        c.tx = btx;
        c.seglen = bseg;
        c.bps = bbps;
        c.ms = best;
        rc = build_class(b, int(k));
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (rc != LBM_OK) return rc;
    if (plan) lbm_batch_get_plan(b, plan);
    return LBM_OK;
}

}  // extern "C"
