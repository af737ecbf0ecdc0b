// C ABI of the phase-field WMRT lattice Boltzmann library (declared in
// include/lbm.h): parameter validation, device memory, stream binding and
// dispatch to the per-lattice kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.cuh"

extern template struct lbm::Launch<lbm::D2Q9, lbm::StoreF32>;
extern template struct lbm::Launch<lbm::D2Q9, lbm::StoreF16>;
extern template struct lbm::Launch<lbm::D2Q9, lbm::StoreBF16>;
extern template struct lbm::Launch<lbm::D3Q19, lbm::StoreF32>;
extern template struct lbm::Launch<lbm::D3Q19, lbm::StoreF16>;
extern template struct lbm::Launch<lbm::D3Q19, lbm::StoreBF16>;

using lbm::D2Q9;
using lbm::D3Q19;
using lbm::DevParams;
using lbm::DiagPartial;
using lbm::Launch;
using lbm::StoreBF16;
using lbm::StoreF16;
using lbm::StoreF32;

// Calls fn with a default-constructed Launch<lattice, storage> of the context.
template <class Fn>
static cudaError_t with_launch(int D, int storage, Fn fn)
{
    if (D == 2) {
        if (storage == 1) return fn(Launch<D2Q9, StoreF16>{});
        if (storage == 2) return fn(Launch<D2Q9, StoreBF16>{});
        return fn(Launch<D2Q9, StoreF32>{});
    }
    if (storage == 1) return fn(Launch<D3Q19, StoreF16>{});
    if (storage == 2) return fn(Launch<D3Q19, StoreBF16>{});
    return fn(Launch<D3Q19, StoreF32>{});
}

struct lbm_ctx {
    lbm_params p;
    DevParams dp;
    int Q, D;
    int64_t N;
    cudaStream_t stream;
    int device;
    lbm::Buffers b;
    lbm::FusedGeom geom;            // work decomposition of the fused step
    int fused_blocks = 0;
    float* face = nullptr;          // phi_in, u_in of the inlet plane
    DiagPartial* diag_part = nullptr;
    DiagPartial* diag_res = nullptr;
    int diag_nparts = 0;
    float* staging = nullptr;       // float32 planes of kStageSets populations for checkpoints
    float* fieldbuf = nullptr;      // in-place layout: (D + 2) N floats staging the fields
    float* outold = nullptr;        // in-place layout: outlet plane kept for the outlet rule
    float* fref = nullptr;          // float16 storage: f reference of each plane of the march axis
    bool ref_set = false;           // fref holds the references of the current encoding
    float* uadv = nullptr;          // prescribed velocity of lbm_advect_phase (host input copied here)
    int* ccl = nullptr;             // jet post-processing scratch: labels, sizes, lo, hi (4 N ints)
    int* ccl_list = nullptr;        // (size, lo, hi) of the components, count at the end
    size_t elem = 4;                // bytes per stored population value
    bool initialised = false;
    // kernel timing: 4 events per recorded step (before phi, after phi,
    // after the collide-stream kernel, after the face kernels)
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    // lbm_step replays kStepGraph steps as one CUDA graph, captured on first
    // use for each assignment of the allocations to A and B (f and g swap
    // together in a step; lbm_advect_phase swaps g alone), on a private
    // stream, and launched on the context's stream
    cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    void* f0 = nullptr;             // the f and g allocations that start as A
    void* g0 = nullptr;
    cudaStream_t cap = nullptr;
    bool no_graphs = false;         // a capture was refused: launch step by step
    // in-step diagnostics (diag_every): steps since the state was set, and
    // the last record
    int64_t step_count = 0;
    int64_t last_diag_step = -1;
    lbm_diag_out last_diag{};
    std::string err;
};

constexpr int64_t kStepGraph = 16;  // steps per graph replay (even: A and B, or the in-place
                                    // layout's parity, end where they began)
constexpr int kStagePops = 4;       // populations converted per pass of a checkpoint

static thread_local std::string g_create_err;

static int fail(lbm_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

static int cuda_fail(lbm_ctx* c, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, m);
}

#define LBM_CUDA(ctx, call)                                              \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);       \
    } while (0)

static int validate(const lbm_params* p, std::string& why)
{
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) { why = "lattice must be 0 (D2Q9) or 1 (D3Q19)"; return -1; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { why = "grid sizes must be >= 1"; return -1; }
    if (p->lattice == LBM_D2Q9 && p->nz != 1) { why = "D2Q9 needs nz == 1"; return -1; }
    if (p->nx > 65535 * 128 || p->ny > 65535 || p->nz > 65535) { why = "grid too large for the launch shape"; return -1; }
    {
        const int64_t nxp = (int64_t(p->nx) + 31) / 32 * 32, Q = p->lattice == LBM_D2Q9 ? 9 : 19;
        if (Q * nxp * p->ny * p->nz > int64_t(UINT32_MAX)) {
            why = "grid too large: population element indices are 32-bit (Q * nodes with rows padded to 32 < 2^32)";
            return -1;
        }
    }
    if (!(p->rho_L > 0 && p->rho_H > 0 && p->tau_H > 0)) { why = "rho_L, rho_H, tau_H must be > 0"; return -1; }
    if (!(p->mu_ratio >= 0)) { why = "mu_ratio must be >= 0 (0: tau_L as given)"; return -1; }
    if (!(p->mu_ratio > 0 || p->tau_L > 0)) { why = "tau_L must be > 0 when mu_ratio is 0"; return -1; }
    // an interface narrower than two lattice units is not resolved by the
    // isotropic stencils of eq:gradient_phi / eq:laplacian_phi
    if (!(p->W >= 2)) { why = "W (interface width) must be >= 2 lattice units"; return -1; }
    if (!(p->mobility > 0 && p->sigma >= 0)) { why = "mobility must be > 0 and sigma >= 0"; return -1; }
    if (p->diag_every < 0) { why = "diag_every must be >= 0"; return -1; }
    if (p->layout != 0 && p->layout != 1) { why = "layout must be 0 (A/B) or 1 (in place)"; return -1; }
    if (p->visc_model != 0 && p->visc_model != 1) { why = "visc_model must be 0 or 1"; return -1; }
    if (p->storage < 0 || p->storage > 2) { why = "storage must be 0 (float32), 1 (float16) or 2 (bfloat16)"; return -1; }
    if (!(p->storage_scale >= 0)) { why = "storage_scale must be >= 0"; return -1; }
    if (p->outlet_scheme < 0 || p->outlet_scheme > 2) { why = "outlet_scheme must be 0, 1 or 2"; return -1; }
    const int D = p->lattice == LBM_D2Q9 ? 2 : 3, L = D - 1;
    const int n[3] = {p->nx, p->ny, p->nz};
    auto open_face = [](int b) { return b == LBM_BC_INLET || b == LBM_BC_OUTFLOW; };
    for (int d = 0; d < D; ++d) {
        const int lo = p->bc[2 * d], hi = p->bc[2 * d + 1];
        if (lo < 0 || lo > 4 || hi < 0 || hi > 4) { why = "face condition out of range"; return -1; }
        if ((lo == LBM_BC_PERIODIC) != (hi == LBM_BC_PERIODIC)) { why = "periodic faces must be paired"; return -1; }
        if (lo == LBM_BC_OUTFLOW || hi == LBM_BC_INLET) { why = "inlet only on a low face, outlet only on a high face"; return -1; }
        if (d != L && (open_face(lo) || open_face(hi))) { why = "inlet/outlet only on the last axis"; return -1; }
    }
    if ((p->bc[2 * L] == LBM_BC_INLET || p->bc[2 * L + 1] == LBM_BC_OUTFLOW) && n[L] < 4) {
        why = "open faces need at least 4 nodes along the last axis";
        return -1;
    }
    if (p->bc[2 * L] == LBM_BC_INLET && !(p->inlet_radius >= 0)) { why = "inlet_radius must be >= 0"; return -1; }
    // what enters through the inlet must be able to leave (Sec. 6 jet set-up)
    if (p->bc[2 * L] == LBM_BC_INLET && p->bc[2 * L + 1] != LBM_BC_OUTFLOW) {
        why = "an inlet needs the convective outlet on the opposite face";
        return -1;
    }
    return 0;
}

// tau_L as given, or from the viscosity ratio: mu_X = rho_X tau_X c_s^2, so
// mu_H / mu_L = mu_ratio gives tau_L = tau_H (rho_H / rho_L) / mu_ratio
static double tau_L_of(const lbm_params* p)
{
    return p->mu_ratio > 0 ? p->tau_H * (p->rho_H / p->rho_L) / p->mu_ratio : p->tau_L;
}

static DevParams make_dev(const lbm_params* p, int64_t N)
{
    DevParams d;
    std::memset(&d, 0, sizeof d);
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    d.nxp = (p->nx + 31) / 32 * 32;
    d.Np = int64_t(d.nxp) * p->ny * p->nz;
    for (int i = 0; i < 6; ++i) d.bc[i] = p->bc[i];
    if (p->lattice == LBM_D2Q9) d.bc[4] = d.bc[5] = LBM_BC_PERIODIC;
    d.visc_model = p->visc_model;
    d.outlet_scheme = p->outlet_scheme;
    d.has_slip = 0;
    for (int f = 0; f < (p->lattice == LBM_D2Q9 ? 4 : 6); ++f)
        if (p->bc[f] == LBM_BC_FREESLIP) d.has_slip = 1;
    d.N = N;
    d.rho_L = float(p->rho_L); d.rho_H = float(p->rho_H);
    const double tau_L = tau_L_of(p);
    d.tau_L = float(tau_L); d.tau_H = float(p->tau_H);
    d.mu_L = float(p->rho_L * tau_L / 3.0); d.mu_H = float(p->rho_H * p->tau_H / 3.0);
    d.beta = float(12.0 * p->sigma / p->W);
    d.kappa = float(1.5 * p->sigma * p->W);
    d.inv_W = float(1.0 / p->W);
    d.omega_phi = float(1.0 / (3.0 * p->mobility + 0.5));
    d.gx = float(p->force[0]); d.gy = float(p->force[1]);
    d.gz = p->lattice == LBM_D2Q9 ? 0.0f : float(p->force[2]);
    d.rho_ref = float(p->rho_ref);
    const double sc = p->storage_scale > 0 ? p->storage_scale : 2048.0;
    d.fscale = float(sc);
    d.inv_fscale = float(1.0 / sc);
    return d;
}

static cudaError_t next_event(lbm_ctx* c, cudaEvent_t* ev)
{
    if (c->events_used == c->events.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        c->events.push_back(e);
    }
    *ev = c->events[c->events_used++];
    return cudaEventRecord(*ev, c->stream);
}

static cudaError_t mark_step(void* ctx)
{
    cudaEvent_t ev;
    return next_event(static_cast<lbm_ctx*>(ctx), &ev);
}

static cudaError_t dispatch_step(lbm_ctx* c)
{
    cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
        using Ln = decltype(l);
        if (c->timing) {
            cudaEvent_t ev;
            cudaError_t r = next_event(c, &ev);
            if (r != cudaSuccess) return r;
            return Ln::step_timed(c->dp, c->geom, c->fused_blocks, c->b, c->stream, mark_step, c);
        }
        return Ln::step_fused(c->dp, c->geom, c->fused_blocks, c->b, c->stream);
    });
    if (c->b.inplace) {
        c->b.par ^= 1;
    } else {
        std::swap(c->b.fA, c->b.fB);
        std::swap(c->b.gA, c->b.gB);
    }
    return e;
}

// Capture kStepGraph steps from the current assignment of A and B into
// c->graph[slot].  Nothing runs during the capture; the buffer pointers are
// restored whatever happens.  Returns the CUDA status (the caller falls back
// to single launches of the same kernels when the capture is refused, e.g.
// inside a caller's own global-mode stream capture).
static cudaError_t capture_steps(lbm_ctx* c, int slot)
{
    if (!c->cap) {
        const cudaError_t ec = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        if (ec != cudaSuccess) {
            c->cap = nullptr;
            return ec;
        }
    }
    const lbm::Buffers saved = c->b;
    cudaStream_t user = c->stream;
    c->stream = c->cap;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int64_t s = 0; s < kStepGraph && e == cudaSuccess; ++s) e = dispatch_step(c);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    c->b = saved;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph[slot], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) c->graph[slot] = nullptr;
    return e;
}

// The diagnostics record of a reduction result.
static void fill_diag(const DiagPartial& r, lbm_diag_out* out)
{
    out->sum_phi = r.sum_phi;
    out->sum_p_in = r.sum_p_in;
    out->sum_p_out = r.sum_p_out;
    out->max_speed = r.max_speed;
    out->n_in = r.n_in;
    out->n_out = r.n_out;
    out->finite = r.nonfinite ? 0 : 1;
    out->reserved = 0;
    out->dp_laplace = (r.n_in > 0 && r.n_out > 0) ? r.sum_p_in / double(r.n_in) - r.sum_p_out / double(r.n_out) : 0.0;
}

// Entry points for the other translation units of the library.
namespace lbm {
int api_validate(const lbm_params* p, std::string& why) { return validate(p, why); }
DevParams api_make_dev(const lbm_params* p, int64_t N) { return make_dev(p, N); }
void api_set_thread_error(const std::string& msg) { g_create_err = msg; }
void api_fill_diag(const DiagPartial& r, lbm_diag_out* out) { fill_diag(r, out); }
}  // namespace lbm

// The FP64 diagnostics of the current state into *r (synchronises).
static int run_diag(lbm_ctx* c, double phase_eps, DiagPartial* r)
{
    cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
        return decltype(l)::diag(c->dp, c->b, phase_eps, c->diag_part, c->diag_nparts, c->diag_res, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "diag kernels");
    LBM_CUDA(c, cudaMemcpyAsync(r, c->diag_res, sizeof *r, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// nsteps steps: whole graphs of kStepGraph steps (not while kernel timing is
// on: its events are recorded between the launches), then single steps.
static int run_steps(lbm_ctx* c, int64_t nsteps)
{
    while (!c->timing && !c->no_graphs && nsteps >= kStepGraph) {
        const int slot = c->b.inplace ? c->b.par : (c->b.fA == c->f0 ? 0 : 1) | (c->b.gA == c->g0 ? 0 : 2);
        if (!c->graph[slot] && capture_steps(c, slot) != cudaSuccess) {
            cudaGetLastError();                 // a refused capture leaves no sticky error
            c->no_graphs = true;
            break;
        }
        LBM_CUDA(c, cudaGraphLaunch(c->graph[slot], c->stream));
        nsteps -= kStepGraph;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaError_t e = dispatch_step(c);
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernels");
    }
    return LBM_OK;
}

extern "C" {

int lbm_create(const lbm_params* p, void* stream, lbm_ctx** out)
{
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, LBM_ERR_ARG, "params is NULL");
    std::string why;
    if (validate(p, why) != 0) return fail(nullptr, LBM_ERR_ARG, why);

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, LBM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
    c->p = *p;
    c->Q = p->lattice == LBM_D2Q9 ? 9 : 19;
    c->D = p->lattice == LBM_D2Q9 ? 2 : 3;
    c->N = int64_t(p->nx) * p->ny * p->nz;
    c->stream = static_cast<cudaStream_t>(stream);
    cudaGetDevice(&c->device);
    c->dp = make_dev(p, c->N);

    c->elem = p->storage == 0 ? 4 : 2;
    const size_t plane = size_t(c->dp.Np) * c->Q * c->elem;
    c->b.inplace = p->layout == 1 ? 1 : 0;
    c->b.par = 0;
    c->b.fB = c->b.gB = nullptr;
    void** bufs[4] = {&c->b.fA, &c->b.gA, &c->b.fB, &c->b.gB};
    for (int k = 0; k < (c->b.inplace ? 2 : 4); ++k) {
        void** b = bufs[k];
        e = cudaMalloc(b, plane);
        if (e != cudaSuccess) {
            int r = cuda_fail(nullptr, e, "cudaMalloc(populations)");
            lbm_destroy(c);
            return r;
        }
    }
    c->f0 = c->b.fA;
    c->g0 = c->b.gA;
    e = cudaMalloc(reinterpret_cast<void**>(&c->b.phi), size_t(c->N) * sizeof(float));
    const int nface = c->D == 2 ? p->nx : p->nx * p->ny;
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c->face), (2 * size_t(nface) + 1) * sizeof(float));
    c->diag_nparts = 2 * 152;
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c->diag_part), (c->diag_nparts + 1) * sizeof(DiagPartial));
    if (e != cudaSuccess) {
        int r = cuda_fail(nullptr, e, "cudaMalloc");
        lbm_destroy(c);
        return r;
    }
    if (e == cudaSuccess && p->storage == 1) {
        const size_t nm = size_t(c->D == 2 ? p->ny : p->nz);
        e = cudaMalloc(reinterpret_cast<void**>(&c->fref), nm * sizeof(float));
        if (e == cudaSuccess) e = cudaMemset(c->fref, 0, nm * sizeof(float));
    }
    if (e == cudaSuccess && c->b.inplace) {
        e = cudaMalloc(reinterpret_cast<void**>(&c->fieldbuf), size_t(c->N) * (c->D + 2) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c->outold), 2 * size_t(c->Q) * nface * sizeof(float));
    }
    if (e != cudaSuccess) {
        int r = cuda_fail(nullptr, e, "cudaMalloc");
        lbm_destroy(c);
        return r;
    }
    c->diag_res = c->diag_part + c->diag_nparts;
    c->dp.phis = c->b.phi;
    c->dp.outold = c->outold;
    c->dp.fref = c->fref;
    e = with_launch(c->D, p->storage, [&](auto l) {
        return decltype(l)::fused_geom(c->dp, &c->geom, &c->fused_blocks, c->b.inplace != 0);
    });
    if (e != cudaSuccess) {
        int r = cuda_fail(nullptr, e, "fused step set-up");
        lbm_destroy(c);
        return r;
    }
    c->dp.phi_in = c->face;
    c->dp.u_in = c->face + nface;
    c->dp.lam = c->face + 2 * nface;
    const int L = c->D - 1;
    if (p->bc[2 * L] == LBM_BC_INLET) {
        e = c->D == 2 ? Launch<D2Q9, StoreF32>::inlet_profile(c->dp, p->inlet_center[0], 0.0, p->inlet_radius,
                                                               p->W, p->inlet_u, c->face, c->face + nface, c->stream)
                      : Launch<D3Q19, StoreF32>::inlet_profile(c->dp, p->inlet_center[0], p->inlet_center[1],
                                                                p->inlet_radius, p->W, p->inlet_u, c->face,
                                                                c->face + nface, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) {
            int r = cuda_fail(nullptr, e, "inlet profile");
            lbm_destroy(c);
            return r;
        }
    }
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c)
{
    if (!c) return LBM_OK;
    cudaStreamSynchronize(c->stream);
    for (cudaGraphExec_t g : c->graph)
        if (g) cudaGraphExecDestroy(g);
    if (c->cap) cudaStreamDestroy(c->cap);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    cudaFree(c->b.fA); cudaFree(c->b.gA); cudaFree(c->b.fB); cudaFree(c->b.gB);
    cudaFree(c->b.phi); cudaFree(c->face); cudaFree(c->diag_part); cudaFree(c->staging); cudaFree(c->uadv);
    cudaFree(c->fieldbuf); cudaFree(c->outold); cudaFree(c->fref);
    cudaFree(c->ccl); cudaFree(c->ccl_list);
    delete c;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c)
{
    return c ? c->err.c_str() : g_create_err.c_str();
}

int lbm_shape(const lbm_ctx* c, int64_t* n_nodes, int32_t* q)
{
    if (!c) return LBM_ERR_ARG;
    if (n_nodes) *n_nodes = c->N;
    if (q) *q = c->Q;
    return LBM_OK;
}

int lbm_set_timing(lbm_ctx* c, int enable)
{
    if (!c) return LBM_ERR_ARG;
    c->timing = enable != 0;
    return LBM_OK;
}

int lbm_get_timing(lbm_ctx* c, double* ms, int64_t* nsteps)
{
    if (!c || !ms) return LBM_ERR_ARG;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    double acc[3] = {0.0, 0.0, 0.0};
    const size_t nrec = c->events_used / 4;
    for (size_t s = 0; s < nrec; ++s) {
        for (int k = 0; k < 3; ++k) {
            float t = 0.0f;
            LBM_CUDA(c, cudaEventElapsedTime(&t, c->events[4 * s + k], c->events[4 * s + k + 1]));
            acc[k] += t;
        }
    }
    for (int k = 0; k < 3; ++k) ms[k] = acc[k];
    if (nsteps) *nsteps = int64_t(nrec);
    c->events_used = 0;
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c)
{
    if (!c) return LBM_ERR_ARG;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// The device address of page-locked (pinned or registered) host memory, or
// nullptr for any other pointer: kernels then read or write the caller's host
// array directly (over the GPU's host link), with no staging copy.
static const void* host_view(const void* p)
{
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();                 // not a CUDA-known pointer: no sticky error
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

int lbm_init_fields(lbm_ctx* c, const float* phi, const float* u, const float* pstar, int on_device)
{
    if (!c) return LBM_ERR_ARG;
    if (!phi) return fail(c, LBM_ERR_ARG, "phi is NULL");
    if (!on_device) {
        // page-locked host fields: the init kernel reads them in place
        const float* vphi = static_cast<const float*>(host_view(phi));
        const float* vu = static_cast<const float*>(host_view(u));
        const float* vp = static_cast<const float*>(host_view(pstar));
        if (vphi && (!u || vu) && (!pstar || vp)) {
            c->b.par = 0;
            cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
                cudaError_t r = c->fref ? decltype(l)::plane_ref(c->dp, vp, 1.0f, c->fref, c->stream) : cudaSuccess;
                if (r == cudaSuccess) r = decltype(l)::init(c->dp, vphi, vu, vp, c->b.fA, c->b.gA, c->stream);
                if (r == cudaSuccess && c->b.inplace) r = decltype(l)::save_outlet(c->dp, c->b, c->stream);
                return r;
            });
            if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
            LBM_CUDA(c, cudaStreamSynchronize(c->stream));
            c->initialised = true;
            c->ref_set = true;
            c->step_count = 0;
            return LBM_OK;
        }
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t nb = size_t(c->N) * sizeof(float);
    // stage the fields in the f buffer B (Q * elem >= 4 (D + 2) bytes per
    // node), or in the field buffer of the in-place layout
    float* s_phi = c->b.inplace ? c->fieldbuf : static_cast<float*>(c->b.fB);
    float* s_u = s_phi + c->N;
    float* s_p = s_phi + c->N * (1 + c->D);
    LBM_CUDA(c, cudaMemcpyAsync(s_phi, phi, nb, kind, c->stream));
    if (u) LBM_CUDA(c, cudaMemcpyAsync(s_u, u, nb * c->D, kind, c->stream));
    if (pstar) LBM_CUDA(c, cudaMemcpyAsync(s_p, pstar, nb, kind, c->stream));
    c->b.par = 0;                           // the equilibria are written in the natural layout
    cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
        const float* vp = pstar ? s_p : nullptr;
        cudaError_t r = c->fref ? decltype(l)::plane_ref(c->dp, vp, 1.0f, c->fref, c->stream) : cudaSuccess;
        if (r == cudaSuccess) r = decltype(l)::init(c->dp, s_phi, u ? s_u : nullptr, vp, c->b.fA, c->b.gA, c->stream);
        if (r == cudaSuccess && c->b.inplace) r = decltype(l)::save_outlet(c->dp, c->b, c->stream);
        return r;
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    if (!on_device) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->initialised = true;
    c->ref_set = true;
    c->step_count = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t nsteps)
{
    if (!c) return LBM_ERR_ARG;
    if (nsteps < 0) return fail(c, LBM_ERR_ARG, "nsteps < 0");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "lbm_step before lbm_init_fields/lbm_set_populations");
    const int64_t k = c->p.diag_every;
    while (nsteps > 0) {
        // up to the next in-step diagnostic (a12: every k steps)
        const int64_t chunk = k > 0 ? std::min(nsteps, k - c->step_count % k) : nsteps;
        const int r = run_steps(c, chunk);
        if (r != LBM_OK) return r;
        c->step_count += chunk;
        nsteps -= chunk;
        if (k > 0 && c->step_count % k == 0) {
            DiagPartial d;
            const int rd = run_diag(c, 1e-3, &d);
            if (rd != LBM_OK) return rd;
            fill_diag(d, &c->last_diag);
            c->last_diag_step = c->step_count;
            if (d.nonfinite)
                return fail(c, LBM_ERR_DIVERGED, "non-finite populations at step " + std::to_string(c->step_count));
        }
    }
    return LBM_OK;
}

int lbm_diag_last(const lbm_ctx* c, lbm_diag_out* out, int64_t* step)
{
    if (!c || !out) return LBM_ERR_ARG;
    *out = c->last_diag;
    if (step) *step = c->last_diag_step;
    return LBM_OK;
}

int lbm_get_fields(lbm_ctx* c, float* phi, float* u, float* p, int on_device)
{
    if (!c) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "no state");
    if (!on_device && (phi || u || p)) {
        // page-locked host outputs: the fields kernel writes them in place
        float* vphi = static_cast<float*>(const_cast<void*>(host_view(phi)));
        float* vu = static_cast<float*>(const_cast<void*>(host_view(u)));
        float* vp = static_cast<float*>(const_cast<void*>(host_view(p)));
        if ((!phi || vphi) && (!u || vu) && (!p || vp)) {
            cudaError_t e = with_launch(c->D, c->p.storage,
                                        [&](auto l) { return decltype(l)::fields(c->dp, c->b, vphi, vu, vp, c->stream); });
            if (e != cudaSuccess) return cuda_fail(c, e, "fields kernel");
            LBM_CUDA(c, cudaStreamSynchronize(c->stream));
            return LBM_OK;
        }
    }
    // outputs are computed into the f buffer B (or the field buffer of the
    // in-place layout), then copied out
    float* o_phi = c->b.inplace ? c->fieldbuf : static_cast<float*>(c->b.fB);
    float* o_u = o_phi + c->N;
    float* o_p = o_phi + c->N * (1 + c->D);
    cudaError_t e = with_launch(c->D, c->p.storage,
                                [&](auto l) { return decltype(l)::fields(c->dp, c->b, o_phi, o_u, o_p, c->stream); });
    if (e != cudaSuccess) return cuda_fail(c, e, "fields kernel");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t nb = size_t(c->N) * sizeof(float);
    if (phi) LBM_CUDA(c, cudaMemcpyAsync(phi, o_phi, nb, kind, c->stream));
    if (u) LBM_CUDA(c, cudaMemcpyAsync(u, o_u, nb * c->D, kind, c->stream));
    if (p) LBM_CUDA(c, cudaMemcpyAsync(p, o_p, nb, kind, c->stream));
    if (!on_device) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// float32 staging planes (kStagePops N) for checkpoints: the external layout
// is population-major planes, the state is blocked (maybe 16-bit, maybe
// swapped); the sets are converted a few populations at a time
static int ensure_staging(lbm_ctx* c)
{
    if (c->staging) return LBM_OK;
    LBM_CUDA(c, cudaMalloc(reinterpret_cast<void**>(&c->staging), size_t(kStagePops) * c->N * sizeof(float)));
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, float* f, float* g, int on_device)
{
    if (!c) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "no state");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int r = ensure_staging(c);
    if (r != LBM_OK) return r;
    float* outs[2] = {f, g};
    for (int set = 0; set < 2; ++set) {
        if (!outs[set]) continue;
        for (int a0 = 0; a0 < c->Q; a0 += kStagePops) {
            const int a1 = std::min(c->Q, a0 + kStagePops);
            cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
                return decltype(l)::unpack(c->dp, c->b, set, a0, a1, c->staging, c->stream);
            });
            if (e != cudaSuccess) return cuda_fail(c, e, "unpack kernel");
            LBM_CUDA(c, cudaMemcpyAsync(outs[set] + size_t(a0) * c->N, c->staging,
                                        size_t(a1 - a0) * c->N * sizeof(float), kind, c->stream));
        }
    }
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const float* f, const float* g, int on_device)
{
    if (!c) return LBM_ERR_ARG;
    if (!f || !g) return fail(c, LBM_ERR_ARG, "f and g are required");
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int r = ensure_staging(c);
    if (r != LBM_OK) return r;
    const float* ins[2] = {f, g};
    void* dst[2] = {c->b.fA, c->b.gA};
    for (int set = 0; set < 2; ++set) {
        for (int a0 = 0; a0 < c->Q; a0 += kStagePops) {
            const int a1 = std::min(c->Q, a0 + kStagePops);
            LBM_CUDA(c, cudaMemcpyAsync(c->staging, ins[set] + size_t(a0) * c->N,
                                        size_t(a1 - a0) * c->N * sizeof(float), kind, c->stream));
            // a context without a state takes the f references from this
            // state (mean f_0 / w_0 of each plane); one with a state keeps
            // its own, so that restoring a state it wrote is exact
            const bool take_ref = c->fref && !c->ref_set && set == 0 && a0 == 0;
            cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
                cudaError_t r = cudaSuccess;
                if (take_ref) r = decltype(l)::plane_ref(c->dp, c->staging, c->D == 2 ? 2.25f : 3.0f, c->fref, c->stream);
                if (r == cudaSuccess) r = decltype(l)::pack(c->dp, c->staging, set, a0, a1, dst[set], c->stream);
                return r;
            });
            if (e != cudaSuccess) return cuda_fail(c, e, "pack kernel");
        }
    }
    c->b.par = 0;                           // written in the natural layout
    if (c->b.inplace) {
        cudaError_t e = with_launch(c->D, c->p.storage,
                                    [&](auto l) { return decltype(l)::save_outlet(c->dp, c->b, c->stream); });
        if (e != cudaSuccess) return cuda_fail(c, e, "outlet copy");
    }
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->initialised = true;
    c->ref_set = true;
    c->step_count = 0;
    return LBM_OK;
}

int lbm_diag(lbm_ctx* c, double phase_eps, lbm_diag_out* out)
{
    if (!c || !out) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "no state");
    DiagPartial r;
    const int rd = run_diag(c, phase_eps, &r);
    if (rd != LBM_OK) return rd;
    fill_diag(r, out);
    if (r.nonfinite) return fail(c, LBM_ERR_DIVERGED, "non-finite populations");
    return LBM_OK;
}

int lbm_advect_phase(lbm_ctx* c, const float* u, double scale, int64_t nsteps, int on_device)
{
    if (!c) return LBM_ERR_ARG;
    if (!u || nsteps < 0) return fail(c, LBM_ERR_ARG, "advect_phase: u is NULL or nsteps < 0");
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "advect_phase before lbm_init_fields/lbm_set_populations");
    for (int f = 0; f < 2 * c->D; ++f)
        if (c->p.bc[f] != LBM_BC_PERIODIC && c->p.bc[f] != LBM_BC_WALL && c->p.bc[f] != LBM_BC_FREESLIP)
            return fail(c, LBM_ERR_ARG, "advect_phase: faces must be periodic, walls or free slip");
    if (c->b.inplace) return fail(c, LBM_ERR_ARG, "advect_phase: needs layout 0 (two copies)");
    const float* ud = u;
    if (!on_device) {
        if (!c->uadv) LBM_CUDA(c, cudaMalloc(reinterpret_cast<void**>(&c->uadv), size_t(c->N) * c->D * sizeof(float)));
        LBM_CUDA(c, cudaMemcpyAsync(c->uadv, u, size_t(c->N) * c->D * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        ud = c->uadv;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
            return decltype(l)::advect(c->dp, c->b, ud, float(scale), c->stream);
        });
        if (e != cudaSuccess) return cuda_fail(c, e, "advect kernels");
        std::swap(c->b.gA, c->b.gB);
    }
    if (!on_device) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_jet_stats(lbm_ctx* c, double threshold, int32_t max_drops, double* drop_volumes, lbm_jet_stats_out* out)
{
    if (!c || !out || max_drops < 0) return LBM_ERR_ARG;
    if (!c->initialised) return fail(c, LBM_ERR_STATE, "no state");
    const int64_t N = c->N;
    if (N > int64_t(INT32_MAX) / 4) return fail(c, LBM_ERR_ARG, "jet_stats: grid too large for its labels");
    constexpr int kCap = 1 << 20;                       // components listed
    if (!c->ccl) LBM_CUDA(c, cudaMalloc(reinterpret_cast<void**>(&c->ccl), 4 * size_t(N) * sizeof(int)));
    if (!c->ccl_list) LBM_CUDA(c, cudaMalloc(reinterpret_cast<void**>(&c->ccl_list), (3 * size_t(kCap) + 2) * sizeof(int)));
    int* lab = c->ccl;
    int* size = lab + N;
    int* lo = size + N;
    int* hi = lo + N;
    int* list = c->ccl_list;
    int* count = list + 3 * kCap;
    int* changed = count + 1;
    const unsigned nb = unsigned((N + 255) / 256);
    cudaError_t e = with_launch(c->D, c->p.storage, [&](auto l) {
        using Ln = decltype(l);
        return Ln::phi(c->dp, c->b, c->stream);
    });
    if (e != cudaSuccess) return cuda_fail(c, e, "phi kernel");
    if (c->D == 2) lbm::k_ccl_init<D2Q9><<<nb, 256, 0, c->stream>>>(c->dp, c->b.phi, float(threshold), lab);
    else lbm::k_ccl_init<D3Q19><<<nb, 256, 0, c->stream>>>(c->dp, c->b.phi, float(threshold), lab);
    int rounds = 0;
    for (;; ++rounds) {
        if (rounds >= 100000) return fail(c, LBM_ERR_TIMEOUT, "jet_stats: labels did not converge");
        LBM_CUDA(c, cudaMemsetAsync(changed, 0, sizeof(int), c->stream));
        if (c->D == 2) lbm::k_ccl_hook<D2Q9><<<nb, 256, 0, c->stream>>>(c->dp, lab, changed);
        else lbm::k_ccl_hook<D3Q19><<<nb, 256, 0, c->stream>>>(c->dp, lab, changed);
        lbm::k_ccl_jump<D2Q9><<<nb, 256, 0, c->stream>>>(N, lab);
        int h = 0;
        LBM_CUDA(c, cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (!h) break;
    }
    LBM_CUDA(c, cudaMemsetAsync(size, 0, size_t(N) * sizeof(int), c->stream));
    LBM_CUDA(c, cudaMemsetAsync(lo, 0x7f, size_t(N) * sizeof(int), c->stream));
    LBM_CUDA(c, cudaMemsetAsync(hi, 0xff, size_t(N) * sizeof(int), c->stream));
    LBM_CUDA(c, cudaMemsetAsync(count, 0, sizeof(int), c->stream));
    if (c->D == 2) lbm::k_ccl_stats<D2Q9><<<nb, 256, 0, c->stream>>>(c->dp, lab, size, lo, hi);
    else lbm::k_ccl_stats<D3Q19><<<nb, 256, 0, c->stream>>>(c->dp, lab, size, lo, hi);
    lbm::k_ccl_list<D2Q9><<<nb, 256, 0, c->stream>>>(N, lab, size, lo, hi, kCap, count, list);
    LBM_CUDA(c, cudaGetLastError());
    int ncomp = 0;
    LBM_CUDA(c, cudaMemcpyAsync(&ncomp, count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    const int nlist = ncomp < kCap ? ncomp : kCap;
    std::vector<int> h(3 * size_t(nlist));
    if (nlist) LBM_CUDA(c, cudaMemcpy(h.data(), list, h.size() * sizeof(int), cudaMemcpyDeviceToHost));
    int jet = -1;
    for (int k = 0; k < nlist; ++k)
        if (h[3 * k + 1] == 0 && (jet < 0 || h[3 * k] > h[3 * jet])) jet = k;
    out->n_components = ncomp;
    out->has_jet = jet >= 0 ? 1 : 0;
    out->breakup_length = jet >= 0 ? double(h[3 * jet + 2] + 1) : 0.0;
    int nd = 0;
    double dsum = 0.0, vsum = 0.0;
    for (int k = 0; k < nlist; ++k) {
        if (k == jet) continue;
        const double v = h[3 * k];
        if (drop_volumes && nd < max_drops) drop_volumes[nd] = v;
        ++nd;
        vsum += v;
        dsum += c->D == 2 ? 2.0 * std::sqrt(v / M_PI) : std::cbrt(6.0 * v / M_PI);
    }
    out->n_drops = nd + (ncomp > kCap ? ncomp - kCap : 0);
    out->truncated = (nd > max_drops || ncomp > kCap) ? 1 : 0;
    out->mean_drop_diameter = nd ? dsum / nd : 0.0;
    out->drop_volume = vsum;
    return LBM_OK;
}

int lbm_collide_cells(const lbm_params* p, int64_t n, const float* f, const float* g, const float* phin,
                      float* fs, float* gs, float* out, void* stream)
{
    if (!p || n < 0 || (n > 0 && (!f || !g || !phin || !fs || !gs)))
        return fail(nullptr, LBM_ERR_ARG, "invalid arguments to lbm_collide_cells");
    if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q19) return fail(nullptr, LBM_ERR_ARG, "bad lattice");
    DevParams d = make_dev(p, 1);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = p->lattice == LBM_D2Q9 ? Launch<D2Q9, StoreF32>::collide_cells(d, n, f, g, phin, fs, gs, out, s)
                                           : Launch<D3Q19, StoreF32>::collide_cells(d, n, f, g, phin, fs, gs, out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "collide cells");
    return LBM_OK;
}

}  // extern "C"
