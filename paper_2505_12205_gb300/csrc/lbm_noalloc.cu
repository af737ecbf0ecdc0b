// lbm_diag_noalloc: the FP64 diagnostics of lbm_diag for callers that cannot
// allocate device memory.
//
// lbm_diag runs on a context, whose creation allocates the populations, a phi
// array, the inlet profile and the reduction partials with cudaMalloc.  Some
// callers cannot do that: code running where device allocation is forbidden
// or would break an allocator that must own every byte (a host framework with
// its own caching allocator, an embedded solver in a real-time loop, a
// plug-in that only receives buffers).  They hold the populations in their own
// memory and want the same reductions.  This entry point runs the same kernels
// (k_phi, k_diag, k_diag_final, and k_inlet_profile for an inlet face) with
// all their scratch in one file-scope static __device__ array, so it calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// Limits: grids up to kMaxNodes nodes and inlet planes up to kMaxFace nodes.
// The array (about 8.6 MB) stays allocated on every device that loads the
// library until the process exits.  Every call shares it: each call rewrites
// everything it reads (nothing has to start at zero), and calls that overlap
// on the GPU (concurrent streams, or concurrent host threads on one device)
// race on it.
#include <cstring>
#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_kernels.cuh"

extern template struct lbm::Launch<lbm::D2Q9, lbm::StoreF32>;
extern template struct lbm::Launch<lbm::D3Q19, lbm::StoreF32>;

namespace lbm {
int api_validate(const lbm_params* p, std::string& why);
DevParams api_make_dev(const lbm_params* p, int64_t N);
void api_set_thread_error(const std::string& msg);
void api_fill_diag(const DiagPartial& r, lbm_diag_out* out);
}  // namespace lbm

namespace {

constexpr int64_t kMaxNodes = int64_t(1) << 21;     // 2,097,152 nodes
constexpr int kMaxFace = 1 << 16;                   // 65,536 inlet-plane nodes
// Width of the first reduction pass: a fixed number of blocks, each reducing a
// grid-strided share of the nodes (two per SM of a 152-SM GB300; any value
// gives the same sums up to FP64 rounding order, which stays fixed).
constexpr int kReduceBlocks = 2 * 152;
constexpr size_t kPartFloats = (kReduceBlocks + 1) * sizeof(lbm::DiagPartial) / sizeof(float);
constexpr size_t kScratchFloats = size_t(kMaxNodes) + 2 * size_t(kMaxFace) + kPartFloats;

static_assert(sizeof(lbm::DiagPartial) % sizeof(double) == 0, "partials must stay 8-byte aligned");
static_assert((size_t(kMaxNodes) + 2 * size_t(kMaxFace)) % 2 == 0, "partials must start 8-byte aligned");

// layout: phi [kMaxNodes] | phi_in, u_in [2 * kMaxFace] | partials [kReduceBlocks + 1]
static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_addr[kMaxDevices] = {};

// errors are reported through lbm_last_error(NULL), like those of lbm_create
int fail(int code, const std::string& msg)
{
    lbm::api_set_thread_error(msg);
    return code;
}

// Device address of the static scratch on the current device.  In host code
// g_scratch names a host-side stand-in, so the address is looked up once per
// device (the first call on a device does this; make that first call before
// any stream capture).  The cached address belongs to the device's primary
// context: it is not valid after cudaDeviceReset or under another driver
// context bound to the same device.
int scratch_address(float** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_addr[dev] = static_cast<float*>(p);
    }
    *out = g_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_diag_noalloc(const lbm_params* p, const float* f, const float* g, double phase_eps,
                                lbm_diag_out* out, void* stream)
{
    if (!p || !f || !g || !out) return fail(LBM_ERR_ARG, "lbm_diag_noalloc: NULL argument");
    std::string why;
    // the planes are float32 whatever storage format p names (the layout of
    // lbm_get_populations, which decodes 16-bit states)
    lbm_params pf = *p;
    pf.storage = 0;
    p = &pf;
    if (lbm::api_validate(p, why) != 0) return fail(LBM_ERR_ARG, "lbm_diag_noalloc: " + why);
    const int64_t N = int64_t(p->nx) * p->ny * p->nz;
    const int D = p->lattice == LBM_D2Q9 ? 2 : 3;
    const int64_t nface = D == 2 ? p->nx : int64_t(p->nx) * p->ny;
    const bool inlet = p->bc[2 * (D - 1)] == LBM_BC_INLET;
    if (N > kMaxNodes)
        return fail(LBM_ERR_ARG, "lbm_diag_noalloc: grid of " + std::to_string(N) +
                                     " nodes exceeds its static scratch of " + std::to_string(kMaxNodes) + " nodes");
    if (inlet && nface > kMaxFace)
        return fail(LBM_ERR_ARG, "lbm_diag_noalloc: inlet plane of " + std::to_string(nface) +
                                     " nodes exceeds its static scratch of " + std::to_string(kMaxFace) + " nodes");
    float* base = nullptr;
    int r = scratch_address(&base);
    if (r != LBM_OK) return r;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    lbm::DevParams dp = lbm::api_make_dev(p, N);
    dp.phi_in = base + kMaxNodes;
    dp.u_in = base + kMaxNodes + kMaxFace;
    lbm::DiagPartial* part = reinterpret_cast<lbm::DiagPartial*>(base + kMaxNodes + 2 * kMaxFace);
    lbm::DiagPartial* res = part + kReduceBlocks;
    lbm::Buffers b;
    b.fA = const_cast<float*>(f);
    b.gA = const_cast<float*>(g);
    b.fB = nullptr;
    b.gB = nullptr;
    b.phi = base;

    cudaError_t e = cudaSuccess;
    if (inlet) {
        e = D == 2 ? lbm::Launch<lbm::D2Q9, lbm::StoreF32>::inlet_profile(dp, p->inlet_center[0], 0.0, p->inlet_radius, p->W,
                                                          p->inlet_u, base + kMaxNodes,
                                                          base + kMaxNodes + kMaxFace, s)
                   : lbm::Launch<lbm::D3Q19, lbm::StoreF32>::inlet_profile(dp, p->inlet_center[0], p->inlet_center[1],
                                                           p->inlet_radius, p->W, p->inlet_u, base + kMaxNodes,
                                                           base + kMaxNodes + kMaxFace, s);
    }
    if (e == cudaSuccess)
        e = D == 2 ? lbm::Launch<lbm::D2Q9, lbm::StoreF32>::diag_planar(dp, b, phase_eps, part, kReduceBlocks, res, s)
                   : lbm::Launch<lbm::D3Q19, lbm::StoreF32>::diag_planar(dp, b, phase_eps, part, kReduceBlocks, res, s);
    lbm::DiagPartial h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, res, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LBM_ERR_CUDA, std::string("lbm_diag_noalloc: ") + cudaGetErrorString(e));
    lbm::api_fill_diag(h, out);
    if (h.nonfinite) return fail(LBM_ERR_DIVERGED, "lbm_diag_noalloc: non-finite populations");
    return LBM_OK;
}
