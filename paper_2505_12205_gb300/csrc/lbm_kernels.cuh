// sm_103a kernels of the phase-field WMRT lattice Boltzmann step.
//
// State: post-streaming populations f, g in 32-node blocks (see "layout"
// below), double-buffered (A = current state, B = next state).  One time step (Algorithms 1-3 of the paper, fused):
//   k_step_fused  per node: phi = sum_a g_a (eq:phase_field_variable) on the
//                 tile and its halo, isotropic stencils of phi
//                 (eq:gradient_phi, eq:laplacian_phi), material properties,
//                 chemical potential, forces, velocity, g-collision
//                 (eq:lbe_interface), f-collision in moment space
//                 (eq:mrt_collision), then push-streaming into B with periodic
//                 wrap and halfway bounce-back (App. B);
//   k_inlet       velocity + phase-field inlet on the inlet plane of B;
//   k_outlet      convective outlet on the outlet plane of B (reads A and B).
// The host swaps A and B after each step.  k_phi + k_fields / k_diag compute
// the macroscopic fields and diagnostics of a state with the same node code.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <type_traits>

#include "lbm_lattice.cuh"

namespace lbm {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_INLET = 2, BC_OUTFLOW = 3, BC_FREESLIP = 4 };

// Parameters as the kernels use them (float32 arithmetic), passed by value.
struct DevParams {
    int nx, ny, nz;
    int nxp;               // nx rounded up to a multiple of 32 (row pitch of the state)
    int bc[6];
    int visc_model;
    int has_slip;          // some face is free slip
    int outlet_scheme;     // 0 local, 1 maximum, 2 average outlet speed (eq:velocity_options)
    int64_t N;             // nodes
    int64_t Np;            // nodes with the padded rows, nxp * ny * nz
    float rho_L, rho_H, tau_L, tau_H, mu_L, mu_H;
    float beta, kappa;     // eq:beta_kappa_relation
    float inv_W;           // 1 / xi
    float omega_phi;       // 1 / (tau_phi + 1/2), tau_phi = M / c_s^2
    float gx, gy, gz, rho_ref;
    float fscale, inv_fscale;   // power-of-two scale of f in 16-bit storage
    // 16-bit storage: reference of f_a / w_a of each plane of the march axis
    // (z in 3D, y in 2D), one float per plane
    const float* fref;
    // inlet plane profile (face arrays, precomputed in double on the device)
    const float* phi_in;
    const float* u_in;
    float* lam;            // outlet: lambda of the maximum / average schemes (one value)
    // in-place layout: phi of the current state (written by the phi pre-pass)
    // and the outlet plane after the previous step's outlet rule, f then g,
    // [2][Q][nface] float32
    const float* phis;
    float* outold;
};

// ------------------------------------------------------------------ layout
//
// The populations of a set are stored in blocks of 32 nodes along x.  Node
// (x, y, z) has the padded index n = (z ny + y) nxp + x (z = 0 and y the row
// in 2D), and population a of node n is element
//     (n / 32) 32 Q + 32 a + n mod 32
// of the set's array.  A warp of 32 consecutive x reads or writes one
// population of a block as one contiguous row (128 B at float32), the Q rows
// of a block are contiguous (2.4 KB for D3Q19 at float32), so that a tile's
// accesses stay within few DRAM pages, and population a of a node is an
// immediate offset 32 a from population 0.  Element indices are 32-bit
// (Q Np < 2^32 is checked on the host).
__device__ __forceinline__ uint32_t pnode(const DevParams& P, int x, int y, int z)
{
    return (uint32_t(z) * uint32_t(P.ny) + uint32_t(y)) * uint32_t(P.nxp) + uint32_t(x);
}

// element of population 0 of padded node n (population a: + 32 a)
template <class L>
__device__ __forceinline__ uint32_t pel(uint32_t n)
{
    return (n >> 5) * (32u * L::Q) + (n & 31u);
}

// Element of population 0 of node (x, y, z) and the stride between the
// populations of a node: the blocked layout of a state, or (PLANAR) the
// population-major planes pop[a N + node] of the external interface.
template <class L, bool PLANAR>
__device__ __forceinline__ int64_t pop_base(const DevParams& P, int64_t node, int x, int y, int z)
{
    if constexpr (PLANAR) return node;
    else return int64_t(pel<L>(pnode(P, x, y, z)));
}
template <bool PLANAR>
__device__ __forceinline__ int64_t pop_stride(const DevParams& P)
{
    if constexpr (PLANAR) return P.N;
    else return 32;
}

// ---------------------------------------------------------- storage formats
//
// Arithmetic is float32 throughout; the populations may be stored in 16 bits
// to halve the bytes a step moves.  Each 16-bit value is normalised by the
// population's weight w_a so that one format covers every direction.
//  - f (float16): f_a / w_a = p* + O(u) is stored as its deviation from a
//    reference r of the node's plane along the march axis (z in 3D, y in 2D),
//    (f_a / w_a - r) * fscale, fscale a power of two.  The reference (the
//    plane's mean p* when the context is given its state) removes the
//    hydrostatic part of p*, so the 11-bit mantissa resolves the velocity
//    moments instead of the pressure head.
//  - g (16-bit fixed point, float16 container): g_a / w_a lies in [-1/2, 3/2]
//    (phi in [0, 1] plus O(u) and interface terms) and is stored as the
//    unsigned integer q = rint((g_a / w_a + 1/2) * 65535 / 2), saturated to
//    [0, 65535]: a uniform step of 3.05e-5 in both bulk phases and across the
//    interface, where float16 resolves only near one value.
// Every conversion uses explicitly rounded operations (no contraction into a
// neighbouring multiply-add), so that every kernel that stores or loads a
// population rounds it the same way.  The format's kRef says whether f takes
// the plane reference; formats without it ignore the argument.
//
// T2 holds the values of two x-adjacent nodes (x even), one aligned 2-element
// access; f2 / g2 / ef2 / eg2 convert both, each lane exactly as the scalar
// conversion does, and lo / hi take one node's value out of a pair.
struct StoreF32 {
    using T = float;
    using T2 = float2;
    static constexpr bool kRef = false;
    __device__ static float f(T v, float, float, const DevParams&) { return v; }
    __device__ static float g(T v, float) { return v; }
    __device__ static T ef(float v, float, float, const DevParams&) { return v; }
    __device__ static T eg(float v, float) { return v; }
    __device__ static float2 f2(T2 v, float, float, const DevParams&) { return v; }
    __device__ static float2 g2(T2 v, float) { return v; }
    __device__ static T2 ef2(float2 v, float, float, const DevParams&) { return v; }
    __device__ static T2 eg2(float2 v, float) { return v; }
    __device__ static T lo(T2 v) { return v.x; }
    __device__ static T hi(T2 v) { return v.y; }
};

// g fixed point: step 2 / 65535 of g / w.  Decoding is one integer-to-float
// conversion (exact) and one fma whose constants are w * step (one rounding,
// the same in every kernel) and w / 2 (exact), so it is correctly rounded
// with respect to them.  Encoding maps g / w onto [0, 1] with a saturating
// fma and rounds to the integer with the 1.5 * 2^23 addend: the low 16 bits
// of the sum are q.  Saturation stores a NaN g as q = 0; a diverging state
// still shows in f (float16 keeps NaN and infinity), which the finite checks
// read.
constexpr float kGStep = 2.0f / 65535.0f;

struct StoreF16 {
    using T = __half;
    static constexpr bool kRef = true;
    __device__ static float f(T v, float wa, float r, const DevParams& P)
    {
        return __fmaf_rn(__half2float(v), __fmul_rn(wa, P.inv_fscale), __fmul_rn(wa, r));
    }
    __device__ static T ef(float v, float wa, float r, const DevParams& P)
    {
        return __float2half_rn(__fmaf_rn(v, P.fscale / wa, -__fmul_rn(r, P.fscale)));
    }
    __device__ static float g(T v, float wa)
    {
        return __fmaf_rn(__uint2float_rn(unsigned(__half_as_ushort(v))), __fmul_rn(wa, kGStep), -0.5f * wa);
    }
    __device__ static T eg(float v, float wa)
    {
        const float s = __saturatef(__fmaf_rn(v, 0.5f / wa, 0.25f));
        const float t = __fmaf_rn(s, 65535.0f, 12582912.0f);
        return __ushort_as_half((unsigned short)(__float_as_uint(t) & 0xffffu));
    }
    using T2 = __half2;
    __device__ static float2 f2(T2 v, float wa, float r, const DevParams& P)
    {
        const float c = __fmul_rn(wa, P.inv_fscale), o = __fmul_rn(wa, r);
        return __ffma2_rn(__half22float2(v), make_float2(c, c), make_float2(o, o));
    }
    __device__ static T2 ef2(float2 v, float wa, float r, const DevParams& P)
    {
        const float c = P.fscale / wa, o = -__fmul_rn(r, P.fscale);
        const float2 t = __ffma2_rn(v, make_float2(c, c), make_float2(o, o));
        return __floats2half2_rn(t.x, t.y);
    }
    __device__ static float2 g2(T2 v, float wa)
    {
        const unsigned u = bits(v);
        const float c = __fmul_rn(wa, kGStep), o = -0.5f * wa;
        return __ffma2_rn(make_float2(__uint2float_rn(u & 0xffffu), __uint2float_rn(u >> 16)), make_float2(c, c),
                          make_float2(o, o));
    }
    __device__ static T2 eg2(float2 v, float wa)
    {
        const float k = 0.5f / wa;
        const float2 s = make_float2(__saturatef(__fmaf_rn(v.x, k, 0.25f)), __saturatef(__fmaf_rn(v.y, k, 0.25f)));
        const float2 t = __ffma2_rn(s, make_float2(65535.0f, 65535.0f), make_float2(12582912.0f, 12582912.0f));
        const unsigned u = __byte_perm(__float_as_uint(t.x), __float_as_uint(t.y), 0x5410);
        return __halves2half2(__ushort_as_half((unsigned short)(u & 0xffffu)), __ushort_as_half((unsigned short)(u >> 16)));
    }
    __device__ static T lo(T2 v) { return __low2half(v); }
    __device__ static T hi(T2 v) { return __high2half(v); }
    __device__ static unsigned bits(T2 v)
    {
        return unsigned(__half_as_ushort(__low2half(v))) | (unsigned(__half_as_ushort(__high2half(v))) << 16);
    }
};

// bfloat16 (8-bit mantissa): f as (f_a / w_a) * fscale, g as g_a / w_a - 1/2,
// no plane reference.  Too coarse for the high-density-ratio cases; kept as
// the plain 16-bit float format.
struct StoreBF16 {
    using T = __nv_bfloat16;
    static constexpr bool kRef = false;
    __device__ static float f(T v, float wa, float, const DevParams& P) { return __fmul_rn(__bfloat162float(v), wa * P.inv_fscale); }
    __device__ static float g(T v, float wa) { return __fmaf_rn(wa, __bfloat162float(v), 0.5f * wa); }
    __device__ static T ef(float v, float wa, float, const DevParams& P) { return __float2bfloat16_rn(__fmul_rn(v, P.fscale / wa)); }
    using T2 = __nv_bfloat162;
    __device__ static float2 f2(T2 v, float wa, float r, const DevParams& P)
    {
        return make_float2(f(__low2bfloat16(v), wa, r, P), f(__high2bfloat16(v), wa, r, P));
    }
    __device__ static float2 g2(T2 v, float wa) { return make_float2(g(__low2bfloat16(v), wa), g(__high2bfloat16(v), wa)); }
    __device__ static T2 ef2(float2 v, float wa, float r, const DevParams& P)
    {
        return __halves2bfloat162(ef(v.x, wa, r, P), ef(v.y, wa, r, P));
    }
    __device__ static T2 eg2(float2 v, float wa) { return __halves2bfloat162(eg(v.x, wa), eg(v.y, wa)); }
    __device__ static T lo(T2 v) { return __low2bfloat16(v); }
    __device__ static T hi(T2 v) { return __high2bfloat16(v); }
    __device__ static T eg(float v, float wa) { return __float2bfloat16_rn(__fmaf_rn(v, 1.0f / wa, -0.5f)); }
};

// Coordinate along the march axis (z in 3D, y in 2D) and the f reference of
// that plane for the format S (0 for formats without one).
template <class L>
__device__ __forceinline__ int march(int y, int z)
{
    return (L::D == 3) ? z : y;
}
template <class S>
__device__ __forceinline__ float fref(const DevParams& P, int m)
{
    if constexpr (S::kRef) return __ldg(P.fref + m);
    else return 0.0f;
}

// ------------------------------------------------------------ node physics

// Deviation of the dimensionless distribution from its weight,
// Gamma_a(u) - w_a (eq:dimensionless_distribution, eq:equilibrium).  It is
// formed directly, not as Gamma_a - w_a, so that float32 keeps the small
// velocity-dependent part exactly instead of losing it to the O(w_a) term.
template <class L>
__device__ __forceinline__ float gdev(int a, float ux, float uy, float uz, float uu)
{
    const float eu = float(L::ex(a)) * ux + float(L::ey(a)) * uy + float(L::ez(a)) * uz;
    return L::w(a) * (3.0f * eu + 4.5f * eu * eu - 1.5f * uu);
}

// Equilibria of both sets (eq:equilibrium_function, eq:equilibrium):
// geq_a = phi Gamma_a, feq_a = p* w_a + Gamma_a - w_a.  The rest population
// takes the remainder so that sum_a geq_a = phi and sum_a feq_a = p* hold to
// the rounding of one sum: float32 weights do not add up to exactly 1, and
// without this every collision would create or destroy a little mass.
template <class L>
__device__ __forceinline__ void equilibria(float phi, float pstar, float ux, float uy, float uz,
                                           float (&geq)[L::Q], float (&feq)[L::Q])
{
    const float uu = ux * ux + uy * uy + uz * uz;
    float sg = 0.0f, sf = 0.0f;
#pragma unroll
    for (int a = 1; a < L::Q; ++a) {
        const float d = gdev<L>(a, ux, uy, uz, uu);
        geq[a] = phi * (L::w(a) + d);
        feq[a] = pstar * L::w(a) + d;
        sg += geq[a];
        sf += feq[a];
    }
    geq[0] = phi - sg;
    feq[0] = pstar - sf;
}

// Weight class of a direction: |e_a|^2 (0 rest, 1 axis, 2 diagonal); the
// weights of D2Q9 and D3Q19 are equal within a class.
template <class L>
__host__ __device__ constexpr int wclass(int a)
{
    return L::ex(a) * L::ex(a) + L::ey(a) * L::ey(a) + L::ez(a) * L::ez(a);
}

// Directions whose component along axis d (0 x, 1 y, 2 z) equals sign.
template <class L>
__host__ __device__ constexpr uint32_t dirmask(int d, int sign)
{
    uint32_t m = 0;
    for (int a = 0; a < L::Q; ++a) {
        const int e = d == 0 ? L::ex(a) : d == 1 ? L::ey(a) : L::ez(a);
        if (e == sign) m |= 1u << a;
    }
    return m;
}

// Index of the direction (ex, ey, ez) (-1 if none).
template <class L>
__host__ __device__ constexpr int dir_index(int ex, int ey, int ez)
{
    for (int a = 0; a < L::Q; ++a)
        if (L::ex(a) == ex && L::ey(a) == ey && L::ez(a) == ez) return a;
    return -1;
}

// Direction a with the components of the axes in mask m (bit d: axis d)
// reversed: the specular image of a after free-slip reflections.
template <class L>
__device__ __forceinline__ int mirrored(int a, int m)
{
    const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
    switch (m & 7) {
    case 1: return dir_index<L>(-ex, ey, ez);
    case 2: return dir_index<L>(ex, -ey, ez);
    case 3: return dir_index<L>(-ex, -ey, ez);
    case 4: return dir_index<L>(ex, ey, -ez);
    case 5: return dir_index<L>(-ex, ey, -ez);
    case 6: return dir_index<L>(ex, -ey, -ez);
    case 7: return dir_index<L>(-ex, -ey, -ez);
    default: return a;
    }
}

template <class L>
__host__ __device__ constexpr bool rest_is_stress_free()
{
    for (int k = 0; k < L::NS; ++k)
        if (L::m(k, 0) != 0) return false;
    return true;
}

// e_a . v without multiplications by the zero or unit components (a product
// with 0 cannot be folded away in IEEE arithmetic; accumulators start at -0,
// the identity of addition).
template <class L>
__device__ __forceinline__ float edot(int a, float vx, float vy, float vz)
{
    float s = -0.0f;
    if (L::ex(a)) s = L::ex(a) > 0 ? s + vx : s - vx;
    if (L::ey(a)) s = L::ey(a) > 0 ? s + vy : s - vy;
    if (L::ez(a)) s = L::ez(a) > 0 ? s + vz : s - vz;
    return s;
}

// Arithmetic on the values of one node (V = float) or of two nodes held in
// the two lanes of packed float32 instructions (V = float2).  Every lane
// rounds as the scalar operation does (round to nearest, no contraction:
// a - b as fma(b, -1, a) is the same rounding as the subtraction), so a
// node's result has the same bits in either form.
template <class V>
struct Lanes;
template <>
struct Lanes<float> {
    static __device__ __forceinline__ float s(float a) { return a; }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float neg(float a) { return -a; }
    static __device__ __forceinline__ float rcp(float a) { return 1.0f / a; }
    static __device__ __forceinline__ float clamp01(float a) { return fminf(fmaxf(a, 0.0f), 1.0f); }
    template <class F>
    static __device__ __forceinline__ float map2(float a, float b, F f) { return f(a, b); }
};
template <>
struct Lanes<float2> {
    static __device__ __forceinline__ float2 s(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }
    static __device__ __forceinline__ float2 rcp(float2 a) { return make_float2(1.0f / a.x, 1.0f / a.y); }
    static __device__ __forceinline__ float2 clamp01(float2 a)
    {
        return make_float2(fminf(fmaxf(a.x, 0.0f), 1.0f), fminf(fmaxf(a.y, 0.0f), 1.0f));
    }
    template <class F>
    static __device__ __forceinline__ float2 map2(float2 a, float2 b, F f) { return make_float2(f(a.x, b.x), f(a.y, b.y)); }
};

// e_a . v in the lanes of V
template <class L, class V>
__device__ __forceinline__ V edot_v(int a, V vx, V vy, V vz)
{
    using O = Lanes<V>;
    V s = O::s(-0.0f);
    if (L::ex(a)) s = L::ex(a) > 0 ? O::add(s, vx) : O::sub(s, vx);
    if (L::ey(a)) s = L::ey(a) > 0 ? O::add(s, vy) : O::sub(s, vy);
    if (L::ez(a)) s = L::ez(a) > 0 ? O::add(s, vz) : O::sub(s, vz);
    return s;
}

// a + b and a - b.  One node's (V = float): both in one packed fma,
// fma(b, +-1, a), which rounds each lane as the add and the subtraction do.
template <class V>
__device__ __forceinline__ void sum_diff(V a, V b, V& s, V& d)
{
    if constexpr (std::is_same<V, float>::value) {
        const float2 sd = __ffma2_rn(make_float2(b, b), make_float2(1.0f, -1.0f), make_float2(a, a));
        s = sd.x;
        d = sd.y;
    } else {
        s = Lanes<V>::add(a, b);
        d = Lanes<V>::sub(a, b);
    }
}

// Macroscopic update and collision of one node (V = float) or of two nodes
// (V = float2, one per lane), written as a stream over the populations so
// that no per-population output array has to live in registers:
//   fa(a)   -> f_a,  ga(a) -> g_a   (post-streaming populations)
//   pa(a)   -> phi(x + e_a)          (stencil values; pa(0) = phi(x), the
//                                     node's own sum_a g_a)
//   emit(a, f*_a, g*_a)              (post-collision populations, when collide)
// The directions are taken in opposite pairs (a, abar): sums and differences
// of a pair give the stencil and the moments, and the equilibria of a pair
// share their even part.
// inlet_node: the node lies on the inlet face, where derivatives of phi are
// not evaluated (the inlet is single phase in the paper's treatment), so the
// interfacial forces vanish there.  out (may be null): phi, u_x, u_y, u_z, p.
template <class T>
struct NoDeduce {
    using type = T;
};
template <class L, bool collide, class V = float, class FA, class GA, class PA, class EM>
__device__ __forceinline__ void node_update(const DevParams& P, FA fa, GA ga, PA pa, bool inlet_node,
                                            typename NoDeduce<V>::type* out, EM emit)
{
    using O = Lanes<V>;
    constexpr int Q = L::Q;
    constexpr float W1 = L::w(1);                       // axis weight
    constexpr float W2 = L::w(Q - 1);                   // diagonal weight
    static_assert(wclass<L>(1) == 1 && wclass<L>(Q - 1) == 2, "direction order");
    static_assert(rest_is_stress_free<L>(), "the rest population carries no stress moment");

    const V phi = pa(0);                                // eq:phase_field_variable

    // eq:gradient_phi, eq:laplacian_phi over opposite pairs, per weight class
    // (c / (c_s^2 dx) = 3, 2 c^2 / (c_s^2 dx^2) = 6)
    V gxs[3] = {O::s(-0.0f), O::s(-0.0f), O::s(-0.0f)}, gys[3] = {O::s(-0.0f), O::s(-0.0f), O::s(-0.0f)};
    V gzs[3] = {O::s(-0.0f), O::s(-0.0f), O::s(-0.0f)}, lps[3] = {O::s(-0.0f), O::s(-0.0f), O::s(-0.0f)};
#pragma unroll
    for (int a = 1; a < Q; ++a) {
        if (L::opp(a) < a) continue;
        const int c = wclass<L>(a);
        V sp, dp;
        sum_diff(pa(a), pa(L::opp(a)), sp, dp);
        lps[c] = O::add(lps[c], O::fma(O::s(-2.0f), phi, sp));   // (phi_a - phi) + (phi_abar - phi)
        if (L::ex(a)) gxs[c] = L::ex(a) > 0 ? O::add(gxs[c], dp) : O::sub(gxs[c], dp);
        if (L::ey(a)) gys[c] = L::ey(a) > 0 ? O::add(gys[c], dp) : O::sub(gys[c], dp);
        if (L::ez(a)) gzs[c] = L::ez(a) > 0 ? O::add(gzs[c], dp) : O::sub(gzs[c], dp);
    }
    V dx = O::fma(O::s(3.0f * W2), gxs[2], O::mul(O::s(3.0f * W1), gxs[1]));
    V dy = O::fma(O::s(3.0f * W2), gys[2], O::mul(O::s(3.0f * W1), gys[1]));
    V dz = (L::D == 2) ? O::s(0.0f) : O::fma(O::s(3.0f * W2), gzs[2], O::mul(O::s(3.0f * W1), gzs[1]));
    V lap = O::fma(O::s(6.0f * W2), lps[2], O::mul(O::s(6.0f * W1), lps[1]));
    if (inlet_node) dx = dy = dz = lap = O::s(0.0f);

    // phi clamped inside the material properties only
    const V ph = O::clamp01(phi);
    const V rho = O::fma(ph, O::s(P.rho_H - P.rho_L), O::s(P.rho_L));   // eq:density_interpolation
    const V inv_rho = O::rcp(rho);
    // Every product that feeds a sum is written as an explicit fma: the
    // compiler fuses a packed multiply into a following packed add whatever
    // the contraction setting, so with V = float2 a separate product and sum
    // would round differently from V = float.
    V tau, tau_h;                                       // tau, tau + 1/2
    if (P.visc_model == 1) {
        tau = O::fma(ph, O::s(P.tau_H - P.tau_L), O::s(P.tau_L));   // eq:relaxation_time
        tau_h = O::add(tau, O::s(0.5f));
    } else {
        const V mu = O::fma(ph, O::s(P.mu_H - P.mu_L), O::s(P.mu_L)), c3 = O::mul(O::s(3.0f), inv_rho);
        tau = O::mul(mu, c3);                                       // eq:dynamic_viscosity, nu = c_s^2 tau
        tau_h = O::fma(mu, c3, O::s(0.5f));
    }
    const V s_nu = O::rcp(tau_h);

    // chemical potential (sign reading: 4 beta (phi - phi_L)(phi - phi_H)(phi - phi_0))
    const V mu_phi = O::fma(O::s(-P.kappa), lap,
                            O::mul(O::mul(O::mul(O::s(4.0f * P.beta), phi), O::sub(phi, O::s(1.0f))),
                                   O::sub(phi, O::s(0.5f))));

    // zeroth, first and second moments of f (eq:normalized_pressure) from
    // the pair sums s = f_a + f_abar and differences d = f_a - f_abar
    V pstar, jx = O::s(-0.0f), jy = O::s(-0.0f), jz = O::s(-0.0f);
    V sxx = O::s(-0.0f), syy = O::s(-0.0f), szz = O::s(-0.0f), sxy = O::s(-0.0f), sxz = O::s(-0.0f),
      syz = O::s(-0.0f);
    {
        pstar = fa(0);
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (L::opp(a) < a) continue;
            const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
            V s, d;
            sum_diff(fa(a), fa(L::opp(a)), s, d);
            pstar = O::add(pstar, s);
            if (ex) jx = ex > 0 ? O::add(jx, d) : O::sub(jx, d);
            if (ey) jy = ey > 0 ? O::add(jy, d) : O::sub(jy, d);
            if (ez) jz = ez > 0 ? O::add(jz, d) : O::sub(jz, d);
            if (ex) sxx = O::add(sxx, s);
            if (ey) syy = O::add(syy, s);
            if (ez) szz = O::add(szz, s);
            if (ex * ey) sxy = ex * ey > 0 ? O::add(sxy, s) : O::sub(sxy, s);
            if (ex * ez) sxz = ex * ez > 0 ? O::add(sxz, s) : O::sub(sxz, s);
            if (ey * ez) syz = ey * ez > 0 ? O::add(syz, s) : O::sub(syz, s);
        }
    }
    const float drho = P.rho_H - P.rho_L;                     // eq:density_gradient_phase_field
    const V rx = O::mul(O::s(drho), dx), ry = O::mul(O::s(drho), dy), rz = O::mul(O::s(drho), dz);
    const V cp = O::mul(O::neg(pstar), O::s(1.0f / 3.0f));  // eq:pressure_force
    const V fb = O::sub(rho, O::s(P.rho_ref));              // eq:gravity_force
    V Fx = O::fma(fb, O::s(P.gx), O::fma(cp, rx, O::mul(mu_phi, dx)));   // F_s + F_p + F_b
    V Fy = O::fma(fb, O::s(P.gy), O::fma(cp, ry, O::mul(mu_phi, dy)));
    V Fz = (L::D == 2) ? O::s(0.0f) : O::fma(fb, O::s(P.gz), O::fma(cp, rz, O::mul(mu_phi, dz)));
    const V h_rho = O::mul(O::s(0.5f), inv_rho);
    auto less_p3 = [&](V sd) { return O::fma(pstar, O::s(-1.0f / 3.0f), sd); };   // Pi_dd - p* c_s^2

    // Viscous force, eq:viscous_force_wmrt, with the predictor velocity u0.
    // Second moments of M^-1 S M (f - feq(u0)): the non-equilibrium stress
    // D = Pi(f) - p* c_s^2 I - u0 u0 (the second moment of feq is exactly
    // p* c_s^2 I + u u on D2Q9 and D3Q19); the deviatoric stress rows relax
    // at s_nu and the trace at 1, so the relaxed stress is
    // s_nu D + (1 - s_nu) tr(D) / dim I.
    {
        const V u0x = O::fma(Fx, h_rho, jx), u0y = O::fma(Fy, h_rho, jy);
        const V u0z = (L::D == 2) ? O::s(0.0f) : O::fma(Fz, h_rho, jz);
        const V dxx = O::fma(O::neg(u0x), u0x, less_p3(sxx)), dyy = O::fma(O::neg(u0y), u0y, less_p3(syy));
        const V dzz = (L::D == 2) ? O::s(0.0f) : O::fma(O::neg(u0z), u0z, less_p3(szz));
        const V dxy = O::fma(O::neg(u0x), u0y, sxy);
        const V iso = O::mul(O::mul(O::sub(O::s(1.0f), s_nu), O::add(O::add(dxx, dyy), dzz)), O::s(1.0f / float(L::D)));
        const V txx = O::fma(s_nu, dxx, iso), tyy = O::fma(s_nu, dyy, iso);
        const V txy = O::mul(s_nu, dxy);
        // nu / c_s^2 = tau
        if constexpr (L::D == 2) {
            Fx = O::fma(O::neg(tau), O::fma(txy, ry, O::mul(txx, rx)), Fx);
            Fy = O::fma(O::neg(tau), O::fma(tyy, ry, O::mul(txy, rx)), Fy);
        } else {
            const V dxz = O::fma(O::neg(u0x), u0z, sxz), dyz = O::fma(O::neg(u0y), u0z, syz);
            const V tzz = O::fma(s_nu, dzz, iso), txz = O::mul(s_nu, dxz), tyz = O::mul(s_nu, dyz);
            Fx = O::fma(O::neg(tau), O::fma(txz, rz, O::fma(txy, ry, O::mul(txx, rx))), Fx);
            Fy = O::fma(O::neg(tau), O::fma(tyz, rz, O::fma(tyy, ry, O::mul(txy, rx))), Fy);
            Fz = O::fma(O::neg(tau), O::fma(tzz, rz, O::fma(tyz, ry, O::mul(txz, rx))), Fz);
        }
    }

    // eq:velocity_update
    const V ux = O::fma(Fx, h_rho, jx), uy = O::fma(Fy, h_rho, jy);
    const V uz = (L::D == 2) ? O::s(0.0f) : O::fma(Fz, h_rho, jz);

    if (out) {
        out[0] = phi;
        out[1] = ux;
        out[2] = uy;
        out[3] = uz;
        out[4] = O::mul(O::mul(pstar, rho), O::s(1.0f / 3.0f));
    }
    if constexpr (!collide) {
        return;
    } else {
        const V uu = O::fma(uz, uz, O::fma(uy, uy, O::mul(ux, ux)));

        // g forcing: eq:forcing_term, n = 0 where |grad phi| < 1e-12
        const V gn2 = O::fma(dz, dz, O::fma(dy, dy, O::mul(dx, dx)));
        const V hp = O::sub(phi, O::s(0.5f));
        const float inv_W = P.inv_W;
        const V amp = O::map2(gn2, hp, [inv_W](float g2, float h) {
            return (g2 >= 1e-24f) ? __fmul_rn(__fmul_rn(__fmaf_rn(-4.0f * h, h, 1.0f), inv_W), rsqrtf(g2)) : 0.0f;
        });

        // f: eq:force_term, eq:equilibrium_modified, eq:mrt_collision with
        // M^-1 S M = I - (1 - s_nu) P:
        //   f* = f - M^-1 S M (f - feq + F/2) + F = feq + F/2 + (1 - s_nu) P (f - feq + F/2).
        // The stress-row moments of f - feq + F/2 are combinations of the
        // non-equilibrium stress E = Pi(f) - p* c_s^2 I - u u (F/2 has none).
        const V exx = O::fma(O::neg(ux), ux, less_p3(sxx)), eyy = O::fma(O::neg(uy), uy, less_p3(syy));
        const V ezz = (L::D == 2) ? O::s(0.0f) : O::fma(O::neg(uz), uz, less_p3(szz));
        const V exy = O::fma(O::neg(ux), uy, sxy), exz = O::fma(O::neg(ux), uz, sxz), eyz = O::fma(O::neg(uy), uz, syz);
        V ck[L::NS];
        const V r = O::sub(O::s(1.0f), s_nu);
        if constexpr (L::D == 2) {
            ck[0] = O::mul(r, O::sub(exx, eyy));             // p_xx row of eq:A1
            ck[1] = O::mul(r, exy);                          // p_xy row
        } else {
            ck[0] = O::mul(r, exy);                          // rows 5-9 of eq:A2
            ck[1] = O::mul(r, eyz);
            ck[2] = O::mul(r, exz);
            ck[3] = O::mul(r, O::sub(O::fma(O::s(2.0f), exx, O::neg(eyy)), ezz));
            ck[4] = O::mul(r, O::sub(eyy, ezz));
        }

        // g: eq:equilibrium_with_force, eq:lbe_interface,
        //   g* = g - w_phi (g - geq + F^phi / 2) + F^phi
        //      = (1 - w_phi) g + w_phi geq + (1 - w_phi / 2) F^phi,  F^phi_a = w_a e_a . n
        const float om = P.omega_phi, om1 = 1.0f - om, kph = 1.0f - 0.5f * om;
        // Equilibria (eq:equilibrium_function, eq:equilibrium) with
        // Gamma_a - w_a = w_a (3 e.u + 4.5 (e.u)^2 - 1.5 u.u), whose even part
        // is shared by a and abar: geq_a = phi w_a + phi (Gamma_a - w_a),
        // feq_a = p* w_a + (Gamma_a - w_a).  The rest population (emitted
        // last) takes the remainder so that sum_a geq_a = phi and
        // sum_a feq_a = p* hold to the rounding of one sum: float32 weights do
        // not add up to exactly 1, and without this every collision would
        // create or destroy mass.
        const V phw1 = O::mul(phi, O::s(W1)), phw2 = O::mul(phi, O::s(W2));
        const V uw1 = O::mul(O::s(-1.5f * W1), uu), uw2 = O::mul(O::s(-1.5f * W2), uu);
        const float kw1 = kph * W1, kw2 = kph * W2;
        const V fr = O::mul(O::s(1.5f), inv_rho);          // F_a / 2 = 1.5 w_a e_a . F / rho
        V sg = O::s(-0.0f), sf = O::s(-0.0f);
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            if (L::opp(a) < a) continue;
            const int b = L::opp(a);
            const bool diag = wclass<L>(a) == 2;
            const float W = diag ? W2 : W1;
            const V eu = edot_v<L>(a, ux, uy, uz);
            const V even = O::fma(O::mul(O::s(4.5f * W), eu), eu, diag ? uw2 : uw1);
            const V da = O::fma(O::s(3.0f * W), eu, even), db = O::fma(O::s(-3.0f * W), eu, even);
            // F^phi_a (1 - w_phi / 2) = (e_a . grad phi) amp w_a (1 - w_phi / 2)
            const V fph = O::mul(O::mul(edot_v<L>(a, dx, dy, dz), amp), O::s(diag ? kw2 : kw1));
            const V ef = O::mul(edot_v<L>(a, Fx, Fy, Fz), fr);          // F_a / 2 = ef w_a
            V proj = O::s(-0.0f);
#pragma unroll
            for (int k = 0; k < L::NS; ++k)
                if (L::m(k, a)) proj = O::fma(O::s(L::rw(k, a)), ck[k], proj);
            const V phw = diag ? phw2 : phw1;
            if constexpr (std::is_same<V, float>::value) {
                // one node: a and b in the two lanes of packed operations,
                // each lane the operation of the general form below
                const float2 d2 = __ffma2_rn(make_float2(eu, eu), make_float2(3.0f * W, -3.0f * W), make_float2(even, even));
                const float2 geq2 = __ffma2_rn(make_float2(phi, phi), d2, make_float2(phw, phw));
                const float2 feq2 = __ffma2_rn(make_float2(pstar, pstar), make_float2(W, W), d2);
                sg = O::add(sg, geq2.x);
                sf = O::add(sf, feq2.x);
                sg = O::add(sg, geq2.y);
                sf = O::add(sf, feq2.y);
                const float2 fo2 = __fadd2_rn(feq2, __ffma2_rn(make_float2(ef, ef), make_float2(W, -W), make_float2(proj, proj)));
                const float2 gi2 = __ffma2_rn(make_float2(om, om), geq2, make_float2(fph, O::neg(fph)));
                const float2 go2 = __ffma2_rn(make_float2(om1, om1), make_float2(ga(a), ga(b)), gi2);
                emit(a, fo2.x, go2.x);
                emit(b, fo2.y, go2.y);
                continue;
            }
            {
                const V geq = O::fma(phi, da, phw);
                const V feq = O::fma(pstar, O::s(W), da);
                sg = O::add(sg, geq);
                sf = O::add(sf, feq);
                emit(a, O::add(feq, O::fma(ef, O::s(W), proj)), O::fma(O::s(om1), ga(a), O::fma(O::s(om), geq, fph)));
            }
            {
                const V geq = O::fma(phi, db, phw);
                const V feq = O::fma(pstar, O::s(W), db);
                sg = O::add(sg, geq);
                sf = O::add(sf, feq);
                emit(b, O::add(feq, O::fma(ef, O::s(-W), proj)), O::fma(O::s(om1), ga(b), O::fma(O::s(om), geq, O::neg(fph))));
            }
        }
        emit(0, O::sub(pstar, sf), O::fma(O::s(om1), ga(0), O::mul(O::s(om), O::sub(phi, sg))));
    }
}

// Array form of node_update for the kernels that hold a node in registers.
template <class L, bool collide>
__device__ __forceinline__ void node_update(const DevParams& P, float (&f)[L::Q], float (&g)[L::Q],
                                            const float (&phin)[L::Q], bool inlet_node, float* out)
{
    float fo[L::Q], go[L::Q];
    node_update<L, collide>(
        P, [&](int a) { return f[a]; }, [&](int a) { return g[a]; }, [&](int a) { return phin[a]; },
        inlet_node, out, [&](int a, float fs, float gs) { fo[a] = fs; go[a] = gs; });
    if (collide) {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            f[a] = fo[a];
            g[a] = go[a];
        }
    }
}

// ----------------------------------------------------------- face mapping

// Neighbour coordinate along one axis for the phi stencil: periodic -> wrap,
// wall/outlet -> clamp (zero normal gradient), inlet -> flag (phi_in).
__device__ __forceinline__ int map_phi(int v, int n, int bclo, int bchi, bool& inlet)
{
    if (v < 0) {
        if (bclo == BC_PERIODIC) return v + n;
        if (bclo == BC_INLET) inlet = true;
        return 0;
    }
    if (v >= n) {
        if (bchi == BC_PERIODIC) return v - n;
        return n - 1;
    }
    return v;
}

// phi at the (possibly out-of-range) node (xx, yy, mm) of the march
// coordinate mm from a phi array of the state, with the ghost rules of the
// faces (the values phi_at forms from g).
template <class L>
__device__ __forceinline__ float phi_ghost(const DevParams& P, const float* __restrict__ phi, int xx, int yy,
                                           int mm)
{
    bool inlet = false;
    const int x = map_phi(xx, P.nx, P.bc[0], P.bc[1], inlet);
    if (L::D == 3) {
        const int y = map_phi(yy, P.ny, P.bc[2], P.bc[3], inlet);
        const int m = map_phi(mm, P.nz, P.bc[4], P.bc[5], inlet);
        if (inlet) return P.phi_in[y * P.nx + x];
        return phi[(int64_t(m) * P.ny + y) * P.nx + x];
    }
    const int m = map_phi(mm, P.ny, P.bc[2], P.bc[3], inlet);
    if (inlet) return P.phi_in[x];
    return phi[int64_t(m) * P.nx + x];
}

// ------------------------------------------------------ in-place (AA) layout
//
// With one copy per set, a step alternates two forms (k_step_fused STEP_EVEN
// and STEP_ODD).  After an odd step (and after initialisation) the state is
// natural: the post-streaming population a of node x is in x's slot a.  After
// an even step it is swapped: each node's post-collision population a sits
// in its own slot abar, so the post-streaming population a of node x is the
// upstream node x - e_a's slot abar -- or, where x - e_a lies beyond a face,
// what the face rule gives: behind a wall or an open face, node x's own slot
// a (the reflected population of halfway bounce-back; at open faces the face
// rules overwrite it); across free-slip faces, the tangential neighbour's
// mirrored population (eq:free_slip_f/g).  par = 1 marks the swapped state.

// Element holding the post-streaming population a of node (x, y, z).  In
// 16-bit storage the value there is encoded with the f reference of the
// plane of (x, y, z), the node it belongs to after streaming, whichever
// node's slot holds it.
template <class L>
__device__ __forceinline__ uint32_t post_el(const DevParams& P, int x, int y, int z, int a, int par)
{
    const uint32_t e0 = pel<L>(pnode(P, x, y, z));
    if (!par || a == 0) return e0 + 32u * uint32_t(a);
    const int pos[3] = {x, y, z};
    const int len[3] = {P.nx, P.ny, P.nz};
    const int e[3] = {L::ex(a), L::ey(a), L::ez(a)};
    int s[3] = {x, y, z}, m = 0;
    bool own = false;
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
        s[d] = pos[d] - e[d];
        if (s[d] < 0 || s[d] >= len[d]) {
            const int bc = P.bc[2 * d + (s[d] < 0 ? 0 : 1)];
            if (bc == BC_PERIODIC) s[d] = s[d] < 0 ? s[d] + len[d] : s[d] - len[d];
            else if (bc == BC_FREESLIP) { s[d] = pos[d]; m |= 1 << d; }
            else own = true;
        }
    }
    if (own) return e0 + 32u * uint32_t(a);
    return pel<L>(pnode(P, s[0], s[1], s[2])) + 32u * uint32_t(L::opp(mirrored<L>(a, m)));
}

// ---------------------------------------------------------------- kernels

// phi = sum_a g_a of every node into phi[node] (unpadded node order); par:
// the state is swapped (in-place layout after an even step).  This is also
// the phi pre-pass of the in-place step.
template <class L, class S, bool PLANAR>
__global__ void __launch_bounds__(128) k_phi(const __grid_constant__ DevParams P,
                                             const typename S::T* __restrict__ g, int par, float* __restrict__ phi)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = int(i % P.nx), y = int((i / P.nx) % P.ny), z = int(i / (int64_t(P.nx) * P.ny));
    float s = 0.0f;
    if (PLANAR || !par) {
        const int64_t b = pop_base<L, PLANAR>(P, i, x, y, z), st = pop_stride<PLANAR>(P);
#pragma unroll
        for (int a = 0; a < L::Q; ++a) s += S::g(__ldg(g + b + a * st), L::w(a));
    } else {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) s += S::g(__ldg(g + post_el<L>(P, x, y, z, a, 1)), L::w(a));
    }
    phi[i] = s;
}

template <class L>
__device__ __forceinline__ void gather_phi(const DevParams& P, const float* __restrict__ phi, int x, int y,
                                           int z, float (&phin)[L::Q])
{
    const int lastax = L::D - 1;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        bool inlet = false;
        const int xx = map_phi(x + L::ex(a), P.nx, P.bc[0], P.bc[1], inlet);
        const int yy = map_phi(y + L::ey(a), P.ny, P.bc[2], P.bc[3], inlet);
        const int zz = (L::D == 3) ? map_phi(z + L::ez(a), P.nz, P.bc[4], P.bc[5], inlet) : 0;
        if (inlet) {
            const int fidx = (lastax == 1) ? xx : (yy * P.nx + xx);
            phin[a] = P.phi_in[fidx];
        } else {
            phin[a] = __ldg(phi + (int64_t(zz) * P.ny + yy) * P.nx + xx);
        }
    }
}

// ------------------------------------------------- fused step (one pass)
//
// One kernel per time step: phi = sum_a g_a is recomputed on the fly from the
// post-streaming g of the current state, so the separate phi pass and the phi
// array disappear from the step.  A block owns a tile of TX x TY columns of
// the plane normal to the last axis (x-y in 3D, x in 2D) and marches along the
// last axis over a segment of planes, keeping a window of three phi planes of
// the tile plus a one-node halo in shared memory; the next plane's interior g
// populations are staged in shared memory while phi of that plane is formed,
// so every population of the state is read from HBM once per step (the halo
// re-reads hit L2 because neighbouring tiles march the same planes at the
// same time).  Blocks are persistent: work items (tile, segment) are dealt
// round-robin, and the segment count is chosen so every block gets the same
// number of items.
struct FusedGeom {
    int tiles_x, tiles_y, ntiles;
    int nseg, seglen;      // segments of the last axis
    int items;             // ntiles * nseg
    int blocks_even;       // in-place layout: persistent blocks of the even form (0: as the odd form)
};

template <class L, int TX, int TY>
struct FusedCfg {
    static constexpr int EX = TX + 2;
    static constexpr int EY = (L::D == 3) ? TY + 2 : 1;
    static constexpr int EXT = EX * EY;                 // extended tile positions
    static constexpr int NT = TX * ((L::D == 3) ? TY : 1);
    static constexpr size_t smem = sizeof(float) * (3 * EXT + 2 * L::Q * NT);
};

// phi at the (possibly out-of-range) node (xx, yy, mm) of the march
// coordinate mm, with the ghost rules of the faces; stores the node's g into
// stash (NT-strided) when stash is not null.
template <class L, class S>
__device__ __forceinline__ float phi_at(const DevParams& P, const typename S::T* __restrict__ gA, int xx, int yy, int mm,
                                        float* stash, int stride)
{
    bool inlet = false;
    const int x = map_phi(xx, P.nx, P.bc[0], P.bc[1], inlet);
    uint32_t n;
    if (L::D == 3) {
        const int y = map_phi(yy, P.ny, P.bc[2], P.bc[3], inlet);
        const int m = map_phi(mm, P.nz, P.bc[4], P.bc[5], inlet);
        if (inlet) return P.phi_in[y * P.nx + x];
        n = pnode(P, x, y, m);
    } else {
        const int m = map_phi(mm, P.ny, P.bc[2], P.bc[3], inlet);
        if (inlet) return P.phi_in[x];
        n = pnode(P, x, m, 0);
    }
    const typename S::T* gb = gA + pel<L>(n);
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        const float v = S::g(__ldg(gb + 32 * a), L::w(a));
        if (stash) stash[a * stride] = v;
        s += v;
    }
    return s;
}

// Push map of one node and plane of the fused step: element offsets o of
// the steps -1, +1 along each axis (wrapped on periodic faces; a step along y
// or the march axis moves whole 32-node blocks, so its offset is the node
// step times Q), the directions pushed back into the node (walls, open faces:
// the face rules overwrite those), the free-slip directions per axis, and
// the f references of the planes mm - 1, mm, mm + 1 of the march axis.
struct PushMap {
    uint32_t o[3][2];
    uint32_t wall, slip[3], off;
    float r[3];
};

// Element that the push of direction a from the node at element e0 writes
// (eq:streaming_f/g, eq:periodic_f/g, eq:no_slip_f/g, eq:free_slip_f/g):
// the neighbour's slot a (push_plain: no face behind a, the usual case, with
// periodic wraps in the offsets), this node's slot abar (wall or open face),
// or the tangential neighbour's mirrored slot (free slip).
template <class L>
__device__ __forceinline__ uint32_t push_plain(const PushMap& M, uint32_t e0, int a)
{
    uint32_t t = e0;
    if (L::ex(a)) t += M.o[0][L::ex(a) > 0];
    if (L::ey(a)) t += M.o[1][L::ey(a) > 0];
    if (L::D == 3 && L::ez(a)) t += M.o[2][L::ez(a) > 0];
    return t + 32u * a;
}
template <class L>
__device__ __forceinline__ uint32_t push_target(const PushMap& M, uint32_t e0, int a)
{
    const uint32_t bit = 1u << a;
    if (!(M.off & bit)) return push_plain<L>(M, e0, a);
    if (M.wall & bit) return e0 + 32u * L::opp(a);
    const int m = int((M.slip[0] >> a) & 1u) | int((M.slip[1] >> a) & 1u) << 1 | int((M.slip[2] >> a) & 1u) << 2;
    uint32_t t = e0;
    if (L::ex(a) && !(m & 1)) t += M.o[0][L::ex(a) > 0];
    if (L::ey(a) && !(m & 2)) t += M.o[1][L::ey(a) > 0];
    if (L::D == 3 && L::ez(a) && !(m & 4)) t += M.o[2][L::ez(a) > 0];
    return t + 32u * mirrored<L>(a, m);
}
// f reference of the node that the push of direction a reaches (the element
// the push writes belongs to it after streaming): the plane one step along
// the march component of a, or this node's plane where a wall, an open face
// or a free-slip face of the march axis keeps the push in it.
template <class L>
__device__ __forceinline__ float push_ref_plain(const PushMap& M, int a)
{
    return M.r[1 + ((L::D == 3) ? L::ez(a) : L::ey(a))];
}
template <class L>
__device__ __forceinline__ float push_ref(const PushMap& M, int a)
{
    if ((M.wall | M.slip[L::D - 1]) & (1u << a)) return M.r[1];
    return push_ref_plain<L>(M, a);
}

// The in-plane part of a node's push map (x, and y in 3D), invariant along
// the march: the directions behind a wall or open face or a free-slip face at
// the node's x (y), and the element offsets of the steps -1 and +1 along x
// (y).  Along x the offset depends only on the lane x mod 32 (a node
// n = 32 B + r moves to n + s; the offset is taken on the block B = 1), and
// uint32 arithmetic is modular, so the periodic wrap s = -(nx - 1) gives the
// right offset too.  A step along y moves whole blocks.
template <class L>
__device__ __forceinline__ void inplane_push(const DevParams& P, int x, int y, PushMap& H)
{
    constexpr int Q = L::Q;
    H.wall = 0u;
    H.slip[0] = H.slip[1] = H.slip[2] = 0u;
    H.o[0][0] = H.o[0][1] = H.o[1][0] = H.o[1][1] = H.o[2][0] = H.o[2][1] = 0u;
    constexpr int DI = (L::D == 3) ? 2 : 1;
    const int pos[2] = {x, y};
    const int len[2] = {P.nx, P.ny};
#pragma unroll
    for (int d = 0; d < DI; ++d) {
        int sm = -1, sp = 1;
        const int lo = P.bc[2 * d], hi = P.bc[2 * d + 1];
        if (pos[d] == 0) {
            if (lo == BC_PERIODIC) sm = len[d] - 1;
            else if (lo == BC_FREESLIP) H.slip[d] |= dirmask<L>(d, -1);
            else H.wall |= dirmask<L>(d, -1);
        }
        if (pos[d] == len[d] - 1) {
            if (hi == BC_PERIODIC) sp = -(len[d] - 1);
            else if (hi == BC_FREESLIP) H.slip[d] |= dirmask<L>(d, 1);
            else H.wall |= dirmask<L>(d, 1);
        }
        if (d == 0) {
            const uint32_t nx0 = uint32_t(x & 31);
            H.o[0][0] = pel<L>(nx0 + 32u + uint32_t(sm)) - pel<L>(nx0 + 32u);
            H.o[0][1] = pel<L>(nx0 + 32u + uint32_t(sp)) - pel<L>(nx0 + 32u);
        } else {
            H.o[1][0] = uint32_t(sm) * uint32_t(P.nxp) * uint32_t(Q);
            H.o[1][1] = uint32_t(sp) * uint32_t(P.nxp) * uint32_t(Q);
        }
    }
}

// The march-axis part of the push map of plane mm (its offsets, face bits
// and the plane references); M.off is formed from all face bits.
template <class L, class S>
__device__ __forceinline__ void march_push(const DevParams& P, int mm, PushMap& M)
{
    constexpr int d = L::D - 1;                 // the march axis
    const int nm = (L::D == 3) ? P.nz : P.ny;
    const uint32_t nstep = (L::D == 3) ? uint32_t(P.nxp) * uint32_t(P.ny) : uint32_t(P.nxp);
    int sm = -1, sp = 1;                        // node steps in units of the axis
    const int lo = P.bc[2 * d], hi = P.bc[2 * d + 1];
    if (mm == 0) {
        if (lo == BC_PERIODIC) sm = nm - 1;
        else if (lo == BC_FREESLIP) M.slip[d] |= dirmask<L>(d, -1);
        else M.wall |= dirmask<L>(d, -1);
    }
    if (mm == nm - 1) {
        if (hi == BC_PERIODIC) sp = -(nm - 1);
        else if (hi == BC_FREESLIP) M.slip[d] |= dirmask<L>(d, 1);
        else M.wall |= dirmask<L>(d, 1);
    }
    M.o[d][0] = uint32_t(sm) * nstep * uint32_t(L::Q);
    M.o[d][1] = uint32_t(sp) * nstep * uint32_t(L::Q);
    M.off = M.wall | M.slip[0] | M.slip[1] | M.slip[2];
    if constexpr (S::kRef) {
        // a push across a non-periodic face stays in plane mm
        M.r[1] = fref<S>(P, mm);
        M.r[0] = (mm > 0 || lo == BC_PERIODIC) ? fref<S>(P, mm + sm) : M.r[1];
        M.r[2] = (mm < nm - 1 || hi == BC_PERIODIC) ? fref<S>(P, mm + sp) : M.r[1];
    } else {
        M.r[0] = M.r[1] = M.r[2] = 0.0f;
    }
}

// Forms of the fused step.
//  STEP_AB    A/B buffers: each node reads its own slots of A and pushes its
//             post-collision populations into B (face rules on the push).
//  In-place (AA) layout, one copy of each set:
//  STEP_EVEN  reads the node's own slots and writes each post-collision
//             population a into the node's own slot abar (streaming is
//             implicit; no face logic), leaving the state "swapped";
//  STEP_ODD   reads each population where the even step left it (the
//             upstream node's opposite slot, or the face rule; aa_src) and
//             pushes the post-collision populations into their natural slots
//             (the push of STEP_AB), leaving the state natural again.
//  In both, a thread writes exactly the slots it read: the read of population
//  a lands where the push of abar writes.  So no two threads touch one slot.
//  phi comes from the array of the phi pre-pass (k_phi): the g slots of a
//  neighbouring node may already hold post-collision values when another
//  block gets to them.
enum { STEP_AB = 0, STEP_EVEN = 1, STEP_ODD = 2 };

// One work item of the fused step: the tile (x0, y0) over the planes
// [m0, m1) of the march axis.  smem: the phi window [3][EY][EX] followed by
// the stash [2][Q][NT]; every thread of the block calls this.  In the
// in-place forms fA == fB and gA == gB.
template <class L, class S, int TX, int TY, int MODE>
__device__ __forceinline__ void fused_item(const DevParams& P, const typename S::T* fA,
                                           const typename S::T* gA, typename S::T* fB,
                                           typename S::T* gB, int x0, int y0, int m0, int m1,
                                           float* smem)
{
    using Cfg = FusedCfg<L, TX, TY>;
    constexpr int Q = L::Q, EX = Cfg::EX, EXT = Cfg::EXT, NT = Cfg::NT;
    constexpr bool INPLACE = MODE != STEP_AB;
    float* win = smem;                    // [3][EY][EX]
    float* stash = smem + 3 * EXT;        // [2][Q][NT]
    const int tid = threadIdx.x + ((L::D == 3) ? threadIdx.y * TX : 0);
    const int tx = threadIdx.x, ty = (L::D == 3) ? threadIdx.y : 0;
    const int nm = (L::D == 3) ? P.nz : P.ny;       // length of the march axis
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < P.nx && ((L::D == 2) || y < P.ny);

    // push map: the in-plane part once, the march-axis part per plane
    PushMap H;
    inplane_push<L>(P, x, y, H);
    auto push_map = [&](int mm) {
        PushMap M = H;
        march_push<L, S>(P, mm, M);
        return M;
    };
    auto plain_target = [&](const PushMap& M, uint32_t e0, int a) { return push_plain<L>(M, e0, a); };
    auto target = [&](const PushMap& M, uint32_t e0, int a) { return push_target<L>(M, e0, a); };
    auto plain_ref = [&](const PushMap& M, int a) { return push_ref_plain<L>(M, a); };
    auto face_ref = [&](const PushMap& M, int a) { return push_ref<L>(M, a); };

    // phi of plane mm over the extended tile into window slot wslot; the
    // interior g of that plane goes to stash buffer (mm mod 2).  The
    // one-node ring around the tile's nodes inside the grid (wx x wy of
    // them) is enumerated on its own, on the first threads, so that only
    // a few warps take the halo path.
    const int wx = min(TX, P.nx - x0), wy = (L::D == 3) ? min(TY, P.ny - y0) : 1;
    const int nh = (L::D == 3) ? 2 * (wx + 2) + 2 * wy : 2;
    auto fill = [&](int mm, float* wslot, bool keep) {
        float* sbuf = stash + (mm & 1) * Q * NT;
        if (own) {
            float v;
            const bool ingrid = mm >= 0 && mm < nm;
            const uint32_t e0 = ingrid ? pel<L>((L::D == 3) ? pnode(P, x, y, mm) : pnode(P, x, mm, 0)) : 0u;
            if constexpr (!INPLACE) {
                if (ingrid) {       // a plane of the grid: no ghost rule applies
                    // (the same sum, in the same order, as phi_at)
                    const typename S::T* gb = gA + e0;
                    float sacc = 0.0f;
#pragma unroll
                    for (int a = 0; a < Q; ++a) {
                        const float gv = S::g(__ldg(gb + 32 * a), L::w(a));
                        if (keep) sbuf[tid + a * NT] = gv;
                        sacc += gv;
                    }
                    v = sacc;
                } else {
                    v = phi_at<L, S>(P, gA, x, y, mm, keep ? sbuf + tid : nullptr, NT);
                }
            } else {
                if (keep) {         // keep implies a plane of the grid
                    if constexpr (MODE == STEP_EVEN) {
#pragma unroll
                        for (int a = 0; a < Q; ++a) sbuf[tid + a * NT] = S::g(__ldg(gA + e0 + 32 * a), L::w(a));
                    } else {
                        // where the even step left each population (the slot
                        // the push of its opposite writes)
                        const PushMap M = push_map(mm);
                        if (__all_sync(__activemask(), M.off == 0u)) {
#pragma unroll
                            for (int a = 0; a < Q; ++a)
                                sbuf[tid + a * NT] = S::g(__ldg(gA + plain_target(M, e0, L::opp(a))), L::w(a));
                        } else {
#pragma unroll
                            for (int a = 0; a < Q; ++a)
                                sbuf[tid + a * NT] = S::g(__ldg(gA + target(M, e0, L::opp(a))), L::w(a));
                        }
                    }
                }
                v = phi_ghost<L>(P, P.phis, x, y, mm);
            }
            wslot[(ty + ((L::D == 3) ? 1 : 0)) * EX + tx + 1] = v;
        }
        for (int h = tid; h < nh; h += NT) {
            int px, py;
            if (L::D == 2) {
                px = h ? wx + 1 : 0;
                py = 0;
            } else if (h < wx + 2) {
                px = h;
                py = 0;
            } else if (h < 2 * (wx + 2)) {
                px = h - (wx + 2);
                py = wy + 1;
            } else {
                px = ((h - 2 * (wx + 2)) & 1) ? wx + 1 : 0;
                py = 1 + ((h - 2 * (wx + 2)) >> 1);
            }
            const int hx = x0 - 1 + px, hy = (L::D == 3) ? y0 - 1 + py : 0;
            if constexpr (!INPLACE) wslot[py * EX + px] = phi_at<L, S>(P, gA, hx, hy, mm, nullptr, 0);
            else wslot[py * EX + px] = phi_ghost<L>(P, P.phis, hx, hy, mm);
        }
    };

    // window slots of planes m - 1, m, m + 1, rotated after each plane
    float* wlo = win;
    float* wmid = win + EXT;
    float* whi = win + 2 * EXT;
    __syncthreads();
    fill(m0 - 1, wlo, false);
    fill(m0, wmid, true);
    for (int m = m0; m < m1; ++m) {
        fill(m + 1, whi, m + 1 < m1);
        __syncthreads();
        if (own) {
            const float* sbuf = stash + (m & 1) * Q * NT + tid;
            const int z = (L::D == 3) ? m : 0;
            const int yc = (L::D == 3) ? y : m;
            const bool inlet_node = m == 0 && P.bc[(L::D == 3) ? 4 : 2] == BC_INLET;
            const uint32_t e0 = pel<L>(pnode(P, x, yc, z));
            auto ga = [&](int a) { return sbuf[a * NT]; };
            const int ctr = (ty + ((L::D == 3) ? 1 : 0)) * EX + tx + 1;
            auto pa = [&](int a) {
                const int dm = (L::D == 3) ? L::ez(a) : L::ey(a);
                const int dy = (L::D == 3) ? L::ey(a) : 0;
                const float* wslot = dm < 0 ? wlo : (dm > 0 ? whi : wmid);
                return wslot[ctr + dy * EX + L::ex(a)];
            };
            if constexpr (MODE == STEP_EVEN) {
                // in place: own slots in, own opposite slots out
                // the value written into slot abar is the post-streaming
                // population a of the node the A/B push of a reaches, and is
                // encoded with the reference of that node's plane
                const PushMap M = push_map(m);
                auto fa = [&](int a) { return S::f(__ldg(fA + e0 + 32 * a), L::w(a), M.r[1], P); };
                auto swap = [&](int a, float fs, float gs) {
                    const float wa = L::w(a);           // w of a and of its opposite
                    fB[e0 + 32 * L::opp(a)] = S::ef(fs, wa, face_ref(M, a), P);
                    gB[e0 + 32 * L::opp(a)] = S::eg(gs, wa);
                };
                node_update<L, true>(P, fa, ga, pa, inlet_node, nullptr, swap);
            } else {
                const PushMap M = push_map(m);
                // when no node of the warp has a direction behind a face (the
                // usual case) every population takes the plain neighbour
                // offset, with no per-direction test (+2 % float32, +15 %
                // float16 throughput); the two cases are separate copies of
                // the node update
                auto step = [&](auto tgt, auto tref) {
                    auto push = [&](int a, float fs, float gs) {
                        const float wa = L::w(a);
                        const uint32_t t = tgt(M, e0, a);
                        fB[t] = S::ef(fs, wa, tref(M, a), P);
                        gB[t] = S::eg(gs, wa);
                    };
                    if constexpr (MODE == STEP_AB) {
                        auto fa = [&](int a) { return S::f(__ldg(fA + e0 + 32 * a), L::w(a), M.r[1], P); };
                        node_update<L, true>(P, fa, ga, pa, inlet_node, nullptr, push);
                    } else {
                        // population a sits where the push of its opposite
                        // writes, encoded with this node's plane reference
                        auto fa = [&](int a) { return S::f(__ldg(fA + tgt(M, e0, L::opp(a))), L::w(a), M.r[1], P); };
                        node_update<L, true>(P, fa, ga, pa, inlet_node, nullptr, push);
                    }
                };
                if (__all_sync(__activemask(), M.off == 0u)) step(plain_target, plain_ref);
                else step(target, face_ref);
            }
        }
        __syncthreads();
        float* t = wlo;
        wlo = wmid;
        wmid = whi;
        whi = t;
    }
}

// ------------------------------------ fused A/B step, two nodes per thread
//
// The A/B step with each thread holding two x-adjacent nodes (x0 + 2t and
// x0 + 2t + 1) in the two lanes of packed float32 instructions: the node
// update runs once for both (node_update with V = float2), a population of
// both nodes is one aligned 2-element load, and a push that does not move
// along x is one aligned 2-element store (along x the two targets straddle a
// pair boundary and are stored one by one).  Each lane's arithmetic is that
// of fused_item, so the result is the same bits.  The tile is TX x TY nodes
// on (TX / 2) x TY threads; the phi window rows start two columns left of
// the tile, so that the pairs of the tile are 8-byte aligned.
template <class L, int TX, int TY>
struct Fused2Cfg {
    static_assert(TX % 2 == 0, "node pairs");
    static constexpr int EX = TX + 4;                   // columns -2 .. TX + 1
    static constexpr int EY = (L::D == 3) ? TY + 2 : 1;
    static constexpr int EXT = EX * EY;
    static constexpr int NT = TX * ((L::D == 3) ? TY : 1);   // nodes of the tile
    static constexpr int NTH = NT / 2;                        // threads
    static constexpr size_t smem = sizeof(float) * (3 * EXT + 2 * L::Q * NT);
};

template <class L, class S, int TX, int TY>
__device__ __forceinline__ void fused_item2(const DevParams& P, const typename S::T* __restrict__ fA,
                                            const typename S::T* __restrict__ gA, typename S::T* __restrict__ fB,
                                            typename S::T* __restrict__ gB, int x0, int y0, int m0, int m1,
                                            float* smem)
{
    using Cfg = Fused2Cfg<L, TX, TY>;
    using O = Lanes<float2>;
    using T = typename S::T;
    using T2 = typename S::T2;
    constexpr int Q = L::Q, EX = Cfg::EX, EXT = Cfg::EXT, NT = Cfg::NT, NTH = Cfg::NTH;
    float* win = smem;                    // [3][EY][EX]
    float* stash = smem + 3 * EXT;        // [2][Q][NT]
    const int tid = threadIdx.x + ((L::D == 3) ? threadIdx.y * (TX / 2) : 0);
    const int tx = 2 * threadIdx.x, ty = (L::D == 3) ? threadIdx.y : 0;   // tile column of node 0
    const int nm = (L::D == 3) ? P.nz : P.ny;
    const int x = x0 + tx, y = y0 + ty;
    const bool own0 = x < P.nx && ((L::D == 2) || y < P.ny);
    const bool own1 = own0 && x + 1 < P.nx;
    const int nid = ty * TX + tx;                                       // stash column of node 0
    const int wc = (ty + ((L::D == 3) ? 1 : 0)) * EX + tx + 2;          // window index of node 0

    PushMap H0, H1;                       // in-plane push maps of the two nodes
    inplane_push<L>(P, x, y, H0);
    inplane_push<L>(P, x + 1, y, H1);

    // phi of plane mm over the extended tile into window slot wslot, and the
    // interior g of that plane into stash buffer (mm mod 2), as in fused_item
    const int wx = min(TX, P.nx - x0), wy = (L::D == 3) ? min(TY, P.ny - y0) : 1;
    const int nh = (L::D == 3) ? 2 * (wx + 2) + 2 * wy : 2;
    auto fill = [&](int mm, float* wslot, bool keep) {
        float* sbuf = stash + (mm & 1) * Q * NT;
        if (own0) {
            float2 v;
            if (mm >= 0 && mm < nm) {
                const uint32_t e0 = pel<L>((L::D == 3) ? pnode(P, x, y, mm) : pnode(P, x, mm, 0));
                const T2* gb = reinterpret_cast<const T2*>(gA + e0);
                float2 sacc = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int a = 0; a < Q; ++a) {
                    const float2 gv = S::g2(__ldg(gb + 16 * a), L::w(a));
                    if (keep) *reinterpret_cast<float2*>(sbuf + nid + a * NT) = gv;
                    sacc = O::add(sacc, gv);
                }
                v = sacc;
            } else {
                v.x = phi_at<L, S>(P, gA, x, y, mm, keep ? sbuf + nid : nullptr, NT);
                v.y = own1 ? phi_at<L, S>(P, gA, x + 1, y, mm, keep ? sbuf + nid + 1 : nullptr, NT) : 0.0f;
            }
            if (own1) *reinterpret_cast<float2*>(wslot + wc) = v;
            else wslot[wc] = v.x;
        }
        for (int h = tid; h < nh; h += NTH) {
            int px, py;
            if (L::D == 2) {
                px = h ? wx + 1 : 0;
                py = 0;
            } else if (h < wx + 2) {
                px = h;
                py = 0;
            } else if (h < 2 * (wx + 2)) {
                px = h - (wx + 2);
                py = wy + 1;
            } else {
                px = ((h - 2 * (wx + 2)) & 1) ? wx + 1 : 0;
                py = 1 + ((h - 2 * (wx + 2)) >> 1);
            }
            const int hx = x0 - 1 + px, hy = (L::D == 3) ? y0 - 1 + py : 0;
            wslot[py * EX + px + 1] = phi_at<L, S>(P, gA, hx, hy, mm, nullptr, 0);
        }
    };

    float* wlo = win;
    float* wmid = win + EXT;
    float* whi = win + 2 * EXT;
    __syncthreads();
    fill(m0 - 1, wlo, false);
    fill(m0, wmid, true);
    for (int m = m0; m < m1; ++m) {
        fill(m + 1, whi, m + 1 < m1);
        __syncthreads();
        if (own0) {
            const float* sbuf = stash + (m & 1) * Q * NT + nid;
            const int z = (L::D == 3) ? m : 0;
            const int yc = (L::D == 3) ? y : m;
            const bool inlet_node = m == 0 && P.bc[(L::D == 3) ? 4 : 2] == BC_INLET;
            const uint32_t e0 = pel<L>(pnode(P, x, yc, z));
            PushMap M0 = H0, M1 = H1;
            march_push<L, S>(P, m, M0);
            march_push<L, S>(P, m, M1);
            auto ga = [sbuf](int a) { return *reinterpret_cast<const float2*>(sbuf + a * NT); };
            // phi at x + e_a of both nodes from the aligned pairs of the row
            // (A = columns -2, -1 of node 0, B = 0, 1, C = 2, 3)
            auto pa = [wlo, wmid, whi, wc](int a) -> float2 {
                const int dm = (L::D == 3) ? L::ez(a) : L::ey(a);
                const int dy = (L::D == 3) ? L::ey(a) : 0;
                const float* r = (dm < 0 ? wlo : (dm > 0 ? whi : wmid)) + wc + dy * EX;
                const float2 B = *reinterpret_cast<const float2*>(r);
                if (L::ex(a) == 0) return B;
                if (L::ex(a) < 0) {
                    const float2 A = *reinterpret_cast<const float2*>(r - 2);
                    return make_float2(A.y, B.x);
                }
                const float2 C = *reinterpret_cast<const float2*>(r + 2);
                return make_float2(B.y, C.x);
            };
            const T2* fp = reinterpret_cast<const T2*>(fA + e0);
            const float rm = M0.r[1];
            auto fa = [&P, fp, rm](int a) { return S::f2(__ldg(fp + 16 * a), L::w(a), rm, P); };
            // no face behind any direction of the warp's nodes: a push along
            // y or the march axis is one pair store, one along x two stores
            auto push_plain2 = [&P, fB, gB, e0, own1, M0, M1](int a, float2 fs, float2 gs) {
                const float wa = L::w(a);
                const T2 fe = S::ef2(fs, wa, push_ref_plain<L>(M0, a), P), ge = S::eg2(gs, wa);
                const uint32_t t0 = push_plain<L>(M0, e0, a);
                if (L::ex(a) == 0 && own1) {
                    *reinterpret_cast<T2*>(fB + t0) = fe;
                    *reinterpret_cast<T2*>(gB + t0) = ge;
                } else {
                    fB[t0] = S::lo(fe);
                    gB[t0] = S::lo(ge);
                    if (own1) {
                        const uint32_t t1 = (L::ex(a) == 0) ? t0 + 1u : push_plain<L>(M1, e0 + 1u, a);
                        fB[t1] = S::hi(fe);
                        gB[t1] = S::hi(ge);
                    }
                }
            };
            if (__all_sync(__activemask(), (M0.off | M1.off) == 0u)) {
                node_update<L, true, float2>(P, fa, ga, pa, inlet_node, nullptr, push_plain2);
            } else {
                // some node of the warp has a face behind a direction: the two
                // nodes one after the other through the scalar update, each
                // with its own push map (the same arithmetic per node)
#pragma unroll 1
                for (int k = 0; k < 2; ++k) {
                    if (k == 1 && !own1) break;
                    PushMap Mk = k ? H1 : H0;
                    march_push<L, S>(P, m, Mk);
                    const uint32_t ek = e0 + uint32_t(k);
                    auto fak = [&](int a) { return S::f(__ldg(fA + ek + 32 * a), L::w(a), rm, P); };
                    auto gak = [&](int a) { return sbuf[a * NT + k]; };
                    auto pak = [&](int a) {
                        const int dm = (L::D == 3) ? L::ez(a) : L::ey(a);
                        const int dy = (L::D == 3) ? L::ey(a) : 0;
                        return (dm < 0 ? wlo : (dm > 0 ? whi : wmid))[wc + k + dy * EX + L::ex(a)];
                    };
                    auto pushk = [&](int a, float fs, float gs) {
                        const uint32_t t = push_target<L>(Mk, ek, a);
                        fB[t] = S::ef(fs, L::w(a), push_ref<L>(Mk, a), P);
                        gB[t] = S::eg(gs, L::w(a));
                    };
                    node_update<L, true>(P, fak, gak, pak, inlet_node, nullptr, pushk);
                }
            }
        }
        __syncthreads();
        float* t = wlo;
        wlo = wmid;
        wmid = whi;
        whi = t;
    }
}

// phi pre-pass of the in-place step: phi = sum_a g_a of every node into
// P.phis (unpadded node order) from the state in either form (par: swapped).
// One thread per node of an x row (grid: rows y, planes z); interior nodes of
// the swapped form take each population from the upstream node's opposite
// slot by a fixed element offset, nodes on a face through post_el.  The sum
// is taken in the order of k_phi and of the A/B step's phi.
template <class L, class S>
__global__ void __launch_bounds__(128) k_phi_pre(const __grid_constant__ DevParams P,
                                                 const typename S::T* __restrict__ g, int par,
                                                 float* __restrict__ phi)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const uint32_t n = pnode(P, x, y, z);
    const uint32_t e0 = pel<L>(n);
    float s = 0.0f;
    if (!par) {
#pragma unroll
        for (int a = 0; a < L::Q; ++a) s += S::g(__ldg(g + e0 + 32 * a), L::w(a));
    } else {
        // element offsets of the node steps -1 and +1 along each axis, wrapped
        // across periodic faces (along x they depend on the lane x mod 32:
        // taken on the block B = 1, modular uint32 arithmetic); a step beyond
        // any other face goes through post_el (face planes in y and z are
        // whole blocks; in x the two edge lanes)
        const int pos[3] = {x, y, z}, len[3] = {P.nx, P.ny, P.nz};
        const uint32_t r = uint32_t(x & 31), nstep[3] = {1u, uint32_t(P.nxp), uint32_t(P.nxp) * uint32_t(P.ny)};
        uint32_t off[3][2];
        bool open[3][2];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int sm = -1, sp = 1;
            open[d][0] = open[d][1] = false;
            if (d < L::D) {
                if (pos[d] == 0) {
                    if (P.bc[2 * d] == BC_PERIODIC) sm = len[d] - 1;
                    else open[d][0] = true;
                }
                if (pos[d] == len[d] - 1) {
                    if (P.bc[2 * d + 1] == BC_PERIODIC) sp = -(len[d] - 1);
                    else open[d][1] = true;
                }
            }
            if (d == 0) {
                off[0][0] = pel<L>(r + 32u + uint32_t(sm)) - pel<L>(r + 32u);
                off[0][1] = pel<L>(r + 32u + uint32_t(sp)) - pel<L>(r + 32u);
            } else {
                off[d][0] = uint32_t(sm) * nstep[d] * uint32_t(L::Q);
                off[d][1] = uint32_t(sp) * nstep[d] * uint32_t(L::Q);
            }
        }
        const bool any_open = open[0][0] || open[0][1] || open[1][0] || open[1][1] || open[2][0] || open[2][1];
        if (!any_open) {
            // every population from the upstream node by its fixed offset: all
            // loads first, then the sum in the order of k_phi
            typename S::T v[L::Q];
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                uint32_t el = e0 + 32u * uint32_t(L::opp(a));
                if (L::ex(a)) el += off[0][L::ex(a) > 0 ? 0 : 1];
                if (L::ey(a)) el += off[1][L::ey(a) > 0 ? 0 : 1];
                if (L::D == 3 && L::ez(a)) el += off[2][L::ez(a) > 0 ? 0 : 1];
                v[a] = __ldg(g + el);
            }
#pragma unroll
            for (int a = 0; a < L::Q; ++a) s += S::g(v[a], L::w(a));
        } else {
#pragma unroll
            for (int a = 0; a < L::Q; ++a) s += S::g(__ldg(g + post_el<L>(P, x, y, z, a, 1)), L::w(a));
        }
    }
    phi[(int64_t(z) * P.ny + y) * P.nx + x] = s;
}

// Resident blocks per SM: for D3Q19 as many as hold 24 warps (the pair-form
// node update needs up to 85 registers), for D2Q9 as many as hold 32 warps
// (64 registers, no spills).
template <class L, int NT>
constexpr int fused_min_blocks() { return (L::D == 3) ? 768 / NT : 1024 / NT; }

// Tile of the in-place forms and the threads per SM each is compiled for:
// the odd form gathers its populations from 2Q different rows and needs more
// registers per thread than the even form (D3Q19: 128, four warps per SM
// sub-partition, where the even form keeps 80).
template <class L> struct InplaceTile;
template <> struct InplaceTile<D2Q9> { static constexpr int TX = 64, TY = 1, ODD_THREADS = 1024; };
template <> struct InplaceTile<D3Q19> { static constexpr int TX = 32, TY = 4, ODD_THREADS = 512; };
template <class L, int NT, int MODE>
constexpr int inplace_min_blocks()
{
    return MODE == STEP_ODD ? InplaceTile<L>::ODD_THREADS / NT : fused_min_blocks<L, NT>();
}

// The fused step, A/B form: fA, gA -> fB, gB, one node per thread.
template <class L, class S, int TX, int TY>
__global__ void __launch_bounds__(TX *((L::D == 3) ? TY : 1), (fused_min_blocks<L, TX *((L::D == 3) ? TY : 1)>()))
k_step_fused(const __grid_constant__ DevParams P, const FusedGeom G, const typename S::T* __restrict__ fA,
             const typename S::T* __restrict__ gA, typename S::T* __restrict__ fB, typename S::T* __restrict__ gB)
{
    extern __shared__ float smem[];
    const int nm = (L::D == 3) ? P.nz : P.ny;
    for (int item = blockIdx.x; item < G.items; item += gridDim.x) {
        const int tile = item % G.ntiles, seg = item / G.ntiles;
        const int x0 = (tile % G.tiles_x) * TX;
        const int y0 = (L::D == 3) ? (tile / G.tiles_x) * TY : 0;
        const int m0 = seg * G.seglen;
        fused_item<L, S, TX, TY, STEP_AB>(P, fA, gA, fB, gB, x0, y0, m0, min(m0 + G.seglen, nm), smem);
    }
}

// The fused step, A/B form, two nodes per thread (MINB resident blocks).
template <class L, class S, int TX, int TY, int MINB>
__global__ void __launch_bounds__(Fused2Cfg<L, TX, TY>::NTH, MINB)
k_step_fused2(const __grid_constant__ DevParams P, const FusedGeom G, const typename S::T* __restrict__ fA,
              const typename S::T* __restrict__ gA, typename S::T* __restrict__ fB, typename S::T* __restrict__ gB)
{
    extern __shared__ float smem[];
    const int nm = (L::D == 3) ? P.nz : P.ny;
    for (int item = blockIdx.x; item < G.items; item += gridDim.x) {
        const int tile = item % G.ntiles, seg = item / G.ntiles;
        const int x0 = (tile % G.tiles_x) * TX;
        const int y0 = (L::D == 3) ? (tile / G.tiles_x) * TY : 0;
        const int m0 = seg * G.seglen;
        fused_item2<L, S, TX, TY>(P, fA, gA, fB, gB, x0, y0, m0, min(m0 + G.seglen, nm), smem);
    }
}

// The fused step on the in-place layout, form MODE (STEP_EVEN or STEP_ODD):
// one copy f, g of each set, read and written (not restrict-qualified).
template <class L, class S, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX *((L::D == 3) ? TY : 1), (inplace_min_blocks<L, TX *((L::D == 3) ? TY : 1), MODE>()))
k_step_inplace(const __grid_constant__ DevParams P, const FusedGeom G, typename S::T* f, typename S::T* g)
{
    extern __shared__ float smem[];
    const int nm = (L::D == 3) ? P.nz : P.ny;
    for (int item = blockIdx.x; item < G.items; item += gridDim.x) {
        const int tile = item % G.ntiles, seg = item / G.ntiles;
        const int x0 = (tile % G.tiles_x) * TX;
        const int y0 = (L::D == 3) ? (tile / G.tiles_x) * TY : 0;
        const int m0 = seg * G.seglen;
        fused_item<L, S, TX, TY, MODE>(P, f, g, f, g, x0, y0, m0, min(m0 + G.seglen, nm), smem);
    }
}

// ---------------------------------------------------------- batched sweeps
//
// Many independent cases of one lattice and storage format advance together:
// one launch per size class and step, over the class's work list of items
// (case, tile segment).  Blocks are persistent and take items from a counter
// (zeroed before each launch), so that items of unequal size balance
// themselves.  Each case keeps its own populations (the blocked layout above,
// from element offset off of the batch arrays) and its own parameters, which
// the block copies into shared memory per item.  Per node the arithmetic is
// that of k_step_fused, so each case evolves exactly as it would alone.
struct BatchCase {
    DevParams P;       // parameters of the case (P.N = its nodes)
    int64_t off;       // first element of the case's populations in the batch arrays
    FusedGeom G;       // its tiles and segments for the class's tile shape
    int pad;
};

template <class L, class S, int TX, int TY>
__global__ void __launch_bounds__(TX *((L::D == 3) ? TY : 1), (fused_min_blocks<L, TX *((L::D == 3) ? TY : 1)>()))
k_step_batch(const BatchCase* __restrict__ cases, const int2* __restrict__ items, int nitems,
             int* __restrict__ counter, const typename S::T* __restrict__ fA, const typename S::T* __restrict__ gA,
             typename S::T* __restrict__ fB, typename S::T* __restrict__ gB)
{
    constexpr int NT = TX * ((L::D == 3) ? TY : 1);
    static_assert(sizeof(BatchCase) % sizeof(int) == 0, "case descriptors are copied as words");
    extern __shared__ float smem[];
    __shared__ BatchCase sc;
    __shared__ int s_item;
    const int tid = threadIdx.x + ((L::D == 3) ? threadIdx.y * TX : 0);
    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) break;                  // the same for every thread
        const int2 it = items[item];
        const int* src = reinterpret_cast<const int*>(cases + it.x);
        int* dst = reinterpret_cast<int*>(&sc);
        for (int k = tid; k < int(sizeof(BatchCase) / sizeof(int)); k += NT) dst[k] = src[k];
        __syncthreads();
        const int nm = (L::D == 3) ? sc.P.nz : sc.P.ny;
        const int tile = it.y % sc.G.ntiles, seg = it.y / sc.G.ntiles;
        const int x0 = (tile % sc.G.tiles_x) * TX;
        const int y0 = (L::D == 3) ? (tile / sc.G.tiles_x) * TY : 0;
        const int m0 = seg * sc.G.seglen;
        const int64_t off = sc.off;
        fused_item<L, S, TX, TY, STEP_AB>(sc.P, fA + off, gA + off, fB + off, gB + off, x0, y0, m0,
                                          min(m0 + sc.G.seglen, nm), smem);
        __syncthreads();                            // sc and s_item are rewritten next
    }
}

// Velocity inlet (f) and phase-field inlet (g) on the low face of the last
// axis, applied to the post-streaming populations in B (App. B).  The
// velocity rule holds for f' = f + F/2 (eq:velocity_boundary_u) with the force
// the next macroscopic update finds at the node: derivatives of phi are not
// evaluated at the inlet, so F is the body force (rho(phi_in) - rho_ref) g
// (eq:gravity_force).  p* cancels, the tangential excess momentum is shared
// by the two unknowns that carry each tangential component, the phase excess
// by the unknowns with a tangential component.
// par: the state is swapped (in-place layout after an even step); the known
// populations are then read where that layout keeps them, and the unknown
// ones (arriving from beyond the face) sit in the node's own slots in either
// layout.
template <class L, class S>
__device__ __forceinline__ void inlet_node(const DevParams& P, typename S::T* fB, typename S::T* gB, int par, int t)
{
    constexpr int Q = L::Q;
    // the node (t mod nx, t / nx) of the last-axis plane 0
    const int tx = (L::D == 2) ? t : t % P.nx, ty = (L::D == 2) ? 0 : t / P.nx;
    const uint32_t e = (L::D == 2) ? pel<L>(pnode(P, tx, 0, 0)) : pel<L>(pnode(P, tx, ty, 0));
    typename S::T* fn = fB + e;
    typename S::T* gn = gB + e;
    auto src = [&](int a) { return (L::D == 2) ? post_el<L>(P, tx, 0, 0, a, par) : post_el<L>(P, tx, ty, 0, a, par); };
    const float r0 = fref<S>(P, 0);     // the node's plane
    const float phin = P.phi_in[t], un = P.u_in[t];
    const float ux = 0.0f, uy = (L::D == 2) ? un : 0.0f, uz = (L::D == 3) ? un : 0.0f;
    const float uu = un * un;
    // F_a / 2 = 1.5 w_a e_a . F / rho with F = (rho - rho_ref) g, rho of phi_in
    const float rin = fmaf(fminf(fmaxf(phin, 0.0f), 1.0f), P.rho_H - P.rho_L, P.rho_L);
    const float hs = (rin - P.rho_ref) * (1.5f / rin);
    const float hx = hs * P.gx, hy = hs * P.gy, hz = hs * P.gz;
    auto half = [&](int a) { return L::w(a) * (float(L::ex(a)) * hx + float(L::ey(a)) * hy + float(L::ez(a)) * hz); };
    // Gamma_a = w_a + gdev_a; the inlet uses f^eq without p* (it cancels)
    float f[Q], g[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const uint32_t e = src(a);
        f[a] = S::f(fB[e], L::w(a), r0, P);
        g[a] = S::g(gB[e], L::w(a));
    }
    float Mx = 0.0f, My = 0.0f, theta = 0.0f;
    int ndiag = 0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int en = (L::D == 2) ? L::ey(a) : L::ez(a);
        const int t0 = L::ex(a), t1 = (L::D == 2) ? 0 : L::ey(a);
        if (en == 0) {
            const float d = gdev<L>(a, ux, uy, uz, uu);
            const float fneq = (f[a] + half(a)) - d;        // f' - feq (p* cancels)
            if (t0) Mx += float(t0) * fneq;
            if (t1) My += float(t1) * fneq;
            theta += g[a] - phin * (L::w(a) + d);     // eq:excess_density
        } else if (en > 0 && (t0 != 0 || t1 != 0)) {
            ++ndiag;
        }
    }
    const float th_n = theta / float(ndiag);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int en = (L::D == 2) ? L::ey(a) : L::ez(a);
        if (en <= 0) continue;
        const int t0 = L::ex(a), t1 = (L::D == 2) ? 0 : L::ey(a);
        const int ab = L::opp(a);
        const float da = gdev<L>(a, ux, uy, uz, uu), db = gdev<L>(ab, ux, uy, uz, uu);
        const float eM = float(t0) * Mx + float(t1) * My;
        // eq:velocity_boundary_distribution on f' = f + F/2, shifted back
        fn[32 * a] = S::ef(((f[ab] + half(ab)) + (da - db) - 0.5f * eM) - half(a), L::w(a), r0, P);
        const float corr = (t0 != 0 || t1 != 0) ? th_n : 0.0f;
        // eq:unknown_distribution_*: g_a = geq_a - (g_abar - geq_abar) - corr, w_a = w_abar
        gn[32 * a] = S::eg(phin * (2.0f * L::w(a) + da + db) - g[ab] - corr, L::w(a));
    }
}

template <class L, class S>
__global__ void k_inlet(const __grid_constant__ DevParams P, typename S::T* fB, typename S::T* gB, int par)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ((L::D == 2) ? P.nx : P.nx * P.ny)) inlet_node<L, S>(P, fB, gB, par, t);
}

// Outlet speed of the maximum / average schemes of eq:velocity_options: the
// bare first moment of f along the outward normal at layer N-1 after
// streaming, reduced over the layer into *P.lam (one block).
template <class L, class S>
__global__ void __launch_bounds__(256) k_outlet_speed(const __grid_constant__ DevParams P, const typename S::T* __restrict__ fB,
                                                      int par)
{
    __shared__ float red[256];
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    const int nL = (L::D == 2) ? P.ny : P.nz;
    float acc = P.outlet_scheme == 1 ? -3.0e38f : 0.0f;
    const float rM = fref<S>(P, nL - 2);
    for (int t = threadIdx.x; t < nface; t += blockDim.x) {
        const int tx = (L::D == 2) ? t : t % P.nx, ty = (L::D == 2) ? 0 : t / P.nx;
        float U = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            const int en = (L::D == 2) ? L::ey(a) : L::ez(a);
            const uint32_t iM = (L::D == 2) ? post_el<L>(P, tx, nL - 2, 0, a, par) : post_el<L>(P, tx, ty, nL - 2, a, par);
            if (en) U += float(en) * S::f(fB[iM], L::w(a), rM, P);
        }
        acc = P.outlet_scheme == 1 ? fmaxf(acc, U) : acc + U;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            red[threadIdx.x] = P.outlet_scheme == 1 ? fmaxf(red[threadIdx.x], red[threadIdx.x + h])
                                                    : red[threadIdx.x] + red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *P.lam = P.outlet_scheme == 1 ? red[0] : red[0] / float(nface);
}

// Convective outlet on the high face of the last axis (eq:implicit_convective,
// eq:convective_f/g): chi(N, t+1) = (chi(N, t) + lambda chi(N-1, t+1)) / (1 + lambda),
// lambda = clamp(sum_a f_a e_a.n at layer N-1 after streaming, 0, 1).
// INPL: in-place layout (par: swapped state); chi(N, t) comes from the copy
// P.outold the previous outlet rule kept (the step overwrote the state's), and
// the result is written to the state and to that copy (as stored: rounded to
// the storage format, so both layouts blend the same values).  A/B: chi(N, t)
// is A's layer N.
template <class L, class S, bool INPL>
__device__ __forceinline__ void outlet_node(const DevParams& P, const typename S::T* fA, const typename S::T* gA,
                                            typename S::T* fB, typename S::T* gB, int par, int t)
{
    constexpr int Q = L::Q;
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    const int nL = (L::D == 2) ? P.ny : P.nz;
    const int tx = (L::D == 2) ? t : t % P.nx, ty = (L::D == 2) ? 0 : t / P.nx;
    auto atN = [&](int a) { return (L::D == 2) ? post_el<L>(P, tx, nL - 1, 0, a, par) : post_el<L>(P, tx, ty, nL - 1, a, par); };
    auto atM = [&](int a) { return (L::D == 2) ? post_el<L>(P, tx, nL - 2, 0, a, par) : post_el<L>(P, tx, ty, nL - 2, a, par); };
    const float rN = fref<S>(P, nL - 1), rM = fref<S>(P, nL - 2);     // planes of the two layers
    float U = 0.0f;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int en = (L::D == 2) ? L::ey(a) : L::ez(a);
        if (en) U += float(en) * S::f(fB[atM(a)], L::w(a), rM, P);
    }
    const float lam = fminf(fmaxf(P.outlet_scheme ? *P.lam : U, 0.0f), 1.0f);
    const float inv = 1.0f / (1.0f + lam);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const float wa = L::w(a);
        const uint32_t iN = atN(a), iM = atM(a);
        const float fo = INPL ? P.outold[a * nface + t] : S::f(fA[iN], wa, rN, P);
        const float go = INPL ? P.outold[(Q + a) * nface + t] : S::g(gA[iN], wa);
        const float fm = S::f(fB[iM], wa, rM, P), gm = S::g(gB[iM], wa);
        const typename S::T fs = S::ef((fo + lam * fm) * inv, wa, rN, P);
        const typename S::T gs = S::eg((go + lam * gm) * inv, wa);
        fB[iN] = fs;
        gB[iN] = gs;
        if (INPL) {
            P.outold[a * nface + t] = S::f(fs, wa, rN, P);
            P.outold[(Q + a) * nface + t] = S::g(gs, wa);
        }
    }
}

template <class L, class S, bool INPL>
__global__ void k_outlet(const __grid_constant__ DevParams P, const typename S::T* fA, const typename S::T* gA,
                         typename S::T* fB, typename S::T* gB, int par)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ((L::D == 2) ? P.nx : P.nx * P.ny)) outlet_node<L, S, INPL>(P, fA, gA, fB, gB, par, t);
}

// Both open-face rules in one launch (outlet with its local speed): threads
// [0, nface) take the inlet plane, [nface, 2 nface) the outlet plane.  The
// two touch disjoint populations (the last axis has at least 4 nodes), so
// the result equals k_inlet followed by k_outlet.
template <class L, class S, bool INPL>
__global__ void k_faces(const __grid_constant__ DevParams P, const typename S::T* fA, const typename S::T* gA,
                        typename S::T* fB, typename S::T* gB, int par)
{
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nface) inlet_node<L, S>(P, fB, gB, par, t);
    else if (t < 2 * nface) outlet_node<L, S, INPL>(P, fA, gA, fB, gB, par, t - nface);
}

// The outlet plane of the state (decoded) into P.outold: chi(N, t) of the
// next outlet rule on the in-place layout, after initialisation or a restore.
template <class L, class S>
__global__ void k_save_outlet(const __grid_constant__ DevParams P, const typename S::T* __restrict__ f,
                              const typename S::T* __restrict__ g, int par)
{
    constexpr int Q = L::Q;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    if (t >= nface) return;
    const int nL = (L::D == 2) ? P.ny : P.nz;
    const int tx = (L::D == 2) ? t : t % P.nx, ty = (L::D == 2) ? 0 : t / P.nx;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const uint32_t iN = (L::D == 2) ? post_el<L>(P, tx, nL - 1, 0, a, par) : post_el<L>(P, tx, ty, nL - 1, a, par);
        P.outold[a * nface + t] = S::f(f[iN], L::w(a), fref<S>(P, nL - 1), P);
        P.outold[(Q + a) * nface + t] = S::g(g[iN], L::w(a));
    }
}

// Inlet-plane profile, computed once in double so that the nozzle mask is the
// same decision as a double-precision reference makes.
template <class L>
__global__ void k_inlet_profile(int nface, int nx, double cx, double cy, double R, double W, double uj,
                                float* phi_in, float* u_in)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nface) return;
    double r;
    if (L::D == 2) {
        r = fabs(double(t) - cx);
    } else {
        const double dx = double(t % nx) - cx, dy = double(t / nx) - cy;
        r = sqrt(dx * dx + dy * dy);
    }
    phi_in[t] = float(0.5 + 0.5 * tanh(2.0 * (R - r) / W));
    u_in[t] = float(r < R ? uj : 0.0);
}

// Mean of scale * X over each plane m of the march axis into ref[m] (one
// block per plane; each thread sums its strided share in double in node
// order and the block adds the shares in a fixed tree, so the result depends
// only on X).  The plane of node i is i / (nodes per plane) in either
// dimension (z planes of nx ny nodes in 3D, y rows of nx nodes in 2D).
template <class L>
__global__ void __launch_bounds__(256) k_plane_ref(const __grid_constant__ DevParams P, const float* __restrict__ X,
                                                   float scale, float* __restrict__ ref)
{
    __shared__ double red[256];
    const int64_t plane = (L::D == 3) ? int64_t(P.nx) * P.ny : int64_t(P.nx);
    const float* xp = X + int64_t(blockIdx.x) * plane;
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < plane; k += 256) acc += double(xp[k]);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) ref[blockIdx.x] = float(double(scale) * red[0] / double(plane));
}

// Equilibrium initialisation from float32 fields (eq:equilibrium,
// eq:equilibrium_function).
template <class L, class S>
__global__ void k_init(const __grid_constant__ DevParams P, const float* __restrict__ phi,
                       const float* __restrict__ u, const float* __restrict__ pstar, typename S::T* __restrict__ f,
                       typename S::T* __restrict__ g)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const float ux = u ? u[i] : 0.0f, uy = u ? u[P.N + i] : 0.0f;
    const float uz = (u && L::D == 3) ? u[2 * P.N + i] : 0.0f;
    const float ps = pstar ? pstar[i] : 0.0f, ph = phi[i];
    float geq[L::Q], feq[L::Q];
    equilibria<L>(ph, ps, ux, uy, uz, geq, feq);
    const int x = int(i % P.nx), y = int((i / P.nx) % P.ny), z = int(i / (int64_t(P.nx) * P.ny));
    const uint32_t e = pel<L>(pnode(P, x, y, z));
    const float r = fref<S>(P, march<L>(y, z));
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        g[e + 32 * a] = S::eg(geq[a], L::w(a));
        f[e + 32 * a] = S::ef(feq[a], L::w(a), r, P);
    }
}

// Macroscopic fields of the state in A (same device code as the step).
template <class L, class S>
__global__ void __launch_bounds__(128) k_fields(const __grid_constant__ DevParams P,
                                                const typename S::T* __restrict__ fA,
                                                const typename S::T* __restrict__ gA, int par,
                                                const float* __restrict__ phi, float* __restrict__ ophi,
                                                float* __restrict__ ou, float* __restrict__ op)
{
    constexpr int Q = L::Q;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x >= P.nx) return;
    const int64_t N = P.N;
    const int64_t node = (int64_t(z) * P.ny + y) * P.nx + x;
    float f[Q], g[Q], phin[Q], out[5];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const uint32_t e = post_el<L>(P, x, y, z, a, par);
        f[a] = S::f(fA[e], L::w(a), fref<S>(P, march<L>(y, z)), P);
        g[a] = S::g(gA[e], L::w(a));
    }
    gather_phi<L>(P, phi, x, y, z, phin);
    const bool inlet_node = ((L::D == 3) ? z : y) == 0 && P.bc[(L::D == 3) ? 4 : 2] == BC_INLET;
    node_update<L, false>(P, f, g, phin, inlet_node, out);
    if (ophi) ophi[node] = out[0];
    if (ou) {
        ou[node] = out[1];
        ou[N + node] = out[2];
        if (L::D == 3) ou[2 * N + node] = out[3];
    }
    if (op) op[node] = out[4];
}

// Advection of the phase field alone in a prescribed velocity field
// scale * uf (uf: D planes of the external node order): phi stencil from the
// phi array (k_phi), the g collision of eq:lbe_interface with the forcing
// term eq:forcing_term (n = 0 where |grad phi| < 1e-12) and g^eq = phi
// Gamma(u), then push streaming of g into gB (periodic wrap, bounce-back at
// walls).  f is not touched.  One thread per node (a test path, not tuned).
template <class L, class S>
__global__ void __launch_bounds__(128) k_advect(const __grid_constant__ DevParams P, const float* __restrict__ phi,
                                                const float* __restrict__ uf, float scale,
                                                const typename S::T* __restrict__ gA, typename S::T* __restrict__ gB)
{
    constexpr int Q = L::Q;
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = int(i % P.nx), y = int((i / P.nx) % P.ny), z = int(i / (int64_t(P.nx) * P.ny));
    float phin[Q];
    gather_phi<L>(P, phi, x, y, z, phin);
    const uint32_t e0 = pel<L>(pnode(P, x, y, z));
    float g[Q], ph = 0.0f;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        g[a] = S::g(gA[e0 + 32 * a], L::w(a));
        ph += g[a];
    }
    float dx = 0.0f, dy = 0.0f, dz = 0.0f;
#pragma unroll
    for (int a = 1; a < Q; ++a) {
        const float wp = 3.0f * L::w(a) * phin[a];
        dx += float(L::ex(a)) * wp;
        dy += float(L::ey(a)) * wp;
        dz += float(L::ez(a)) * wp;
    }
    const float gn2 = dx * dx + dy * dy + dz * dz;
    const float amp = (gn2 >= 1e-24f) ? (1.0f - 4.0f * (ph - 0.5f) * (ph - 0.5f)) * P.inv_W * rsqrtf(gn2) : 0.0f;
    const float ux = scale * uf[i], uy = scale * uf[P.N + i], uz = (L::D == 3) ? scale * uf[2 * P.N + i] : 0.0f;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float om = P.omega_phi;
    float sg = 0.0f, gs[Q];
#pragma unroll
    for (int a = 1; a < Q; ++a) {
        const float en = amp * (float(L::ex(a)) * dx + float(L::ey(a)) * dy + float(L::ez(a)) * dz);
        const float Fphi = L::w(a) * en;
        const float geq = ph * (L::w(a) + gdev<L>(a, ux, uy, uz, uu));
        sg += geq;
        gs[a] = g[a] - om * (g[a] - geq + 0.5f * Fphi) + Fphi;
    }
    gs[0] = g[0] - om * (g[0] - (ph - sg));
    // push streaming of g
    const int pos[3] = {x, y, z};
    const int len[3] = {P.nx, P.ny, P.nz};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int e[3] = {L::ex(a), L::ey(a), L::ez(a)};
        int t[3], m = 0;
        bool wall = false;
        for (int d = 0; d < 3; ++d) {
            t[d] = pos[d] + e[d];
            if (t[d] < 0 || t[d] >= len[d]) {
                const int bc = P.bc[2 * d + (t[d] < 0 ? 0 : 1)];
                if (bc == BC_PERIODIC) t[d] = (t[d] + len[d]) % len[d];
                else if (bc == BC_FREESLIP) { t[d] = pos[d]; m |= 1 << d; }
                else wall = true;
            }
        }
        const float wa = L::w(a);
        if (wall) gB[e0 + 32 * L::opp(a)] = S::eg(gs[a], wa);
        else gB[pel<L>(pnode(P, t[0], t[1], t[2])) + 32 * mirrored<L>(a, m)] = S::eg(gs[a], wa);
    }
}

// ------------------------------------------------- jet post-processing
//
// Connected components of the liquid phi > threshold (face neighbours,
// periodic wrap across periodic faces) by minimum-label propagation with
// pointer jumping; the host repeats the two passes until no label changes
// (with a bounded number of rounds).  Labels are unpadded node indices; a
// component's label converges to its smallest node index.
template <class L>
__global__ void k_ccl_init(const __grid_constant__ DevParams P, const float* __restrict__ phi, float thr,
                           int* __restrict__ lab)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < P.N) lab[i] = phi[i] > thr ? int(i) : -1;
}

template <class L>
__global__ void k_ccl_hook(const __grid_constant__ DevParams P, int* __restrict__ lab, int* __restrict__ changed)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int li = lab[i];
    if (li < 0) return;
    const int x = int(i % P.nx), y = int((i / P.nx) % P.ny), z = int(i / (int64_t(P.nx) * P.ny));
    const int pos[3] = {x, y, z}, len[3] = {P.nx, P.ny, P.nz};
    const int64_t str[3] = {1, P.nx, int64_t(P.nx) * P.ny};
    int m = li;
    for (int d = 0; d < L::D; ++d)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int q = pos[d] + sgn;
            if (q < 0 || q >= len[d]) {
                if (P.bc[2 * d + (q < 0 ? 0 : 1)] != BC_PERIODIC) continue;
                q = (q + len[d]) % len[d];
            }
            const int lj = lab[i + (q - pos[d]) * str[d]];
            if (lj >= 0 && lj < m) m = lj;
        }
    if (m < li) {
        atomicMin(&lab[li], m);            // hook the root of this label as well
        atomicMin(&lab[i], m);
        *changed = 1;
    }
}

template <class L>
__global__ void k_ccl_jump(int64_t n, int* __restrict__ lab)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int l = lab[i];
    if (l < 0) return;
    for (int k = 0; k < 64 && lab[l] != l && lab[l] >= 0; ++k) l = lab[l];
    lab[i] = l;
}

// Per root: cells, and the smallest / largest coordinate along the last axis.
template <class L>
__global__ void k_ccl_stats(const __grid_constant__ DevParams P, const int* __restrict__ lab, int* __restrict__ size,
                            int* __restrict__ lo, int* __restrict__ hi)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int l = lab[i];
    if (l < 0) return;
    const int m = int((L::D == 3) ? i / (int64_t(P.nx) * P.ny) : (i / P.nx) % P.ny);
    atomicAdd(&size[l], 1);
    atomicMin(&lo[l], m);
    atomicMax(&hi[l], m);
}

// Roots (label == own index) appended to a list of (size, lo, hi).
template <class L>
__global__ void k_ccl_list(int64_t n, const int* __restrict__ lab, const int* __restrict__ size,
                           const int* __restrict__ lo, const int* __restrict__ hi, int cap, int* __restrict__ count,
                           int* __restrict__ list)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n || lab[i] != int(i)) return;
    const int k = atomicAdd(count, 1);
    if (k < cap) {
        list[3 * k] = size[i];
        list[3 * k + 1] = lo[i];
        list[3 * k + 2] = hi[i];
    }
}

// Per-block FP64 partial reductions for lbm_diag.
struct DiagPartial {
    double sum_phi, sum_p_in, sum_p_out, max_speed;
    long long n_in, n_out;
    int nonfinite;
    int pad;
};

template <class L, class S, bool PLANAR>
__global__ void __launch_bounds__(256) k_diag(const __grid_constant__ DevParams P,
                                              const typename S::T* __restrict__ fA,
                                              const typename S::T* __restrict__ gA, int par,
                                              const float* __restrict__ phi, double eps,
                                              DiagPartial* __restrict__ part)
{
    constexpr int Q = L::Q;
    __shared__ double s_phi[256], s_pin[256], s_pout[256], s_max[256];
    __shared__ long long s_nin[256], s_nout[256];
    __shared__ int s_bad[256];
    double a_phi = 0.0, a_pin = 0.0, a_pout = 0.0, a_max = 0.0;
    long long a_nin = 0, a_nout = 0;
    int bad = 0;
    const int64_t N = P.N;
    for (int64_t node = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; node < N;
         node += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(node % P.nx);
        const int y = int((node / P.nx) % P.ny);
        const int z = int(node / (int64_t(P.nx) * P.ny));
        float f[Q], g[Q], phin[Q], out[5];
        const int64_t b = pop_base<L, PLANAR>(P, node, x, y, z), st = pop_stride<PLANAR>(P);
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int64_t e = (!PLANAR && par) ? int64_t(post_el<L>(P, x, y, z, a, 1)) : b + a * st;
            f[a] = S::f(fA[e], L::w(a), fref<S>(P, march<L>(y, z)), P);
            g[a] = S::g(gA[e], L::w(a));
            if (!isfinite(f[a]) || !isfinite(g[a])) bad = 1;
        }
        gather_phi<L>(P, phi, x, y, z, phin);
        const bool inlet_node = ((L::D == 3) ? z : y) == 0 && P.bc[(L::D == 3) ? 4 : 2] == BC_INLET;
        node_update<L, false>(P, f, g, phin, inlet_node, out);
        a_phi += double(out[0]);
        const double sp = sqrt(double(out[1]) * out[1] + double(out[2]) * out[2] + double(out[3]) * out[3]);
        a_max = fmax(a_max, sp);
        if (out[0] >= 1.0 - eps) { a_pin += double(out[4]); ++a_nin; }
        if (out[0] <= eps) { a_pout += double(out[4]); ++a_nout; }
    }
    const int t = threadIdx.x;
    s_phi[t] = a_phi; s_pin[t] = a_pin; s_pout[t] = a_pout; s_max[t] = a_max;
    s_nin[t] = a_nin; s_nout[t] = a_nout; s_bad[t] = bad;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (t < h) {
            s_phi[t] += s_phi[t + h]; s_pin[t] += s_pin[t + h]; s_pout[t] += s_pout[t + h];
            s_max[t] = fmax(s_max[t], s_max[t + h]);
            s_nin[t] += s_nin[t + h]; s_nout[t] += s_nout[t + h]; s_bad[t] |= s_bad[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        DiagPartial r;
        r.sum_phi = s_phi[0]; r.sum_p_in = s_pin[0]; r.sum_p_out = s_pout[0]; r.max_speed = s_max[0];
        r.n_in = s_nin[0]; r.n_out = s_nout[0]; r.nonfinite = s_bad[0]; r.pad = 0;
        part[blockIdx.x] = r;
    }
}

// Final reduction of the partials in a fixed order (one thread: deterministic).
template <class L>
__global__ void k_diag_final(const DiagPartial* __restrict__ part, int nparts, DiagPartial* __restrict__ res)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    DiagPartial r = {0.0, 0.0, 0.0, 0.0, 0, 0, 0, 0};
    for (int i = 0; i < nparts; ++i) {
        r.sum_phi += part[i].sum_phi; r.sum_p_in += part[i].sum_p_in; r.sum_p_out += part[i].sum_p_out;
        r.max_speed = fmax(r.max_speed, part[i].max_speed);
        r.n_in += part[i].n_in; r.n_out += part[i].n_out; r.nonfinite |= part[i].nonfinite;
    }
    *res = r;
}

// Test hook: collision of independent cells, layout [n][Q].
template <class L>
__global__ void k_collide_cells(const __grid_constant__ DevParams P, int64_t n, const float* __restrict__ fi,
                                const float* __restrict__ gi, const float* __restrict__ pin,
                                float* __restrict__ fo, float* __restrict__ go, float* __restrict__ out)
{
    constexpr int Q = L::Q;
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float f[Q], g[Q], phin[Q], o[5];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        f[a] = fi[c * Q + a];
        g[a] = gi[c * Q + a];
        phin[a] = pin[c * Q + a];
    }
    node_update<L, true>(P, f, g, phin, false, o);
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        fo[c * Q + a] = f[a];
        go[c * Q + a] = g[a];
    }
    if (out)
        for (int k = 0; k < 5; ++k) out[c * 5 + k] = o[k];
}

// ------------------------------------------------------ host-side launchers

// Device buffers of a context; the population planes hold S::T values.
// A/B layout: A the current state, B the next.  In-place layout: the state is
// fA, gA alone (fB, gB unused) and par says whether it is swapped.
struct Buffers {
    void *fA, *gA, *fB, *gB;
    float* phi;
    int inplace;
    int par;
};

template <class L, class S>
struct Launch {
    using T = typename S::T;
    // fused single-pass step (k_step_fused + face kernels); geometry from fused_geom
    static cudaError_t step_fused(const DevParams& P, const FusedGeom& G, int nblocks, const Buffers& b,
                                  cudaStream_t s);
    // inplace: size the persistent grid for the in-place kernels
    static cudaError_t fused_geom(const DevParams& P, FusedGeom* G, int* nblocks, bool inplace = false);
    // the outlet plane of the in-place state into P.outold
    static cudaError_t save_outlet(const DevParams& P, const Buffers& b, cudaStream_t s);
    // the same launches as step_fused, with mark(mctx) recording an event
    // after each stage
    using MarkFn = cudaError_t (*)(void*);
    static cudaError_t step_timed(const DevParams& P, const FusedGeom& G, int nblocks, const Buffers& b,
                                  cudaStream_t s, MarkFn mark, void* mctx);
    static cudaError_t init(const DevParams& P, const float* phi, const float* u, const float* pstar, void* f,
                            void* g, cudaStream_t s);
    static cudaError_t fields(const DevParams& P, const Buffers& b, float* ophi, float* ou, float* op,
                              cudaStream_t s);
    static cudaError_t diag(const DevParams& P, const Buffers& b, double eps, DiagPartial* part, int nparts,
                            DiagPartial* res, cudaStream_t s);
    // the same diagnostics of populations in the external population-major
    // planes [Q][N] (f32 planes of the caller)
    static cudaError_t diag_planar(const DevParams& P, const Buffers& b, double eps, DiagPartial* part, int nparts,
                                   DiagPartial* res, cudaStream_t s);
    // populations a0 .. a1-1 of one set of the state <-> float32 planes
    // (checkpoints); gset: the g set; unpack reads the layout of b (A), pack
    // writes the natural layout into dst
    static cudaError_t unpack(const DevParams& P, const Buffers& b, int gset, int a0, int a1, float* out,
                              cudaStream_t s);
    static cudaError_t pack(const DevParams& P, const float* in, int gset, int a0, int a1, void* dst, cudaStream_t s);
    static cudaError_t inlet_profile(const DevParams& P, double cx, double cy, double R, double W, double uj,
                                     float* phi_in, float* u_in, cudaStream_t s);
    static cudaError_t collide_cells(const DevParams& P, int64_t n, const float* f, const float* g,
                                     const float* phin, float* fs, float* gs, float* out, cudaStream_t s);
    // phi = sum_a g_a of the state in A into b.phi (unpadded node order)
    static cudaError_t phi(const DevParams& P, const Buffers& b, cudaStream_t s);
    // f references of 16-bit storage: ref[m] = scale * (mean of X over plane m
    // of the march axis), X float32 in the unpadded node order (NULL: 0)
    static cudaError_t plane_ref(const DevParams& P, const float* X, float scale, float* ref, cudaStream_t s);
    // one step of the phase field alone in the velocity scale * uf (g: A -> B)
    static cudaError_t advect(const DevParams& P, const Buffers& b, const float* uf, float scale, cudaStream_t s);
};

// Tile shapes: 32 x 6 columns in 3D (four 192-thread blocks per SM), 64 nodes
// of a row in 2D (sixteen 64-thread blocks per SM); measured best of
// 32 x {4..8} and {32..256} x 1 on the 3D jet and the 2D Rayleigh-Taylor
// workloads.
template <class L> struct FusedTile;
template <> struct FusedTile<D2Q9> { static constexpr int TX = 64, TY = 1; };
template <> struct FusedTile<D3Q19> { static constexpr int TX = 32, TY = 6; };

// The A/B step of each lattice and storage format: PAIR, two nodes per
// thread (fused_item2) or one (fused_item), the tile and, for pairs, the
// resident blocks per SM (a thread's register budget is 64 K / (threads x
// blocks)).  Measured on the 3D jet and the 2D Rayleigh-Taylor workloads:
// pairs gain with 16-bit storage (9 % on the jet, 14 % on Rayleigh-Taylor,
// fewer instructions per update where the step is bound by issue), not with
// float32, where the step is bound by memory latency and one node per thread
// keeps twice the warps resident.
template <class L, class S> struct ABStep {
    static constexpr bool PAIR = !std::is_same<S, StoreF32>::value;
    static constexpr int TX = PAIR ? 64 : FusedTile<L>::TX;
    static constexpr int TY = (L::D == 2) ? 1 : (PAIR ? 4 : FusedTile<L>::TY);
    static constexpr int MINB = (L::D == 2) ? 20 : 4;
};

template <class L, class S>
cudaError_t Launch<L, S>::fused_geom(const DevParams& P, FusedGeom* G, int* nblocks, bool inplace)
{
    G->blocks_even = 0;
    constexpr int TX = InplaceTile<L>::TX, TY = InplaceTile<L>::TY;
    using AB = ABStep<L, S>;
    constexpr int TX2 = AB::TX, TY2 = AB::TY;
    using Cfg = FusedCfg<L, TX, TY>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (!inplace) {
        // the A/B step of this format: two nodes per thread, or one
        auto occupancy = [&](auto kern, int threads, size_t smem) {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
            if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
            return r;
        };
        if constexpr (AB::PAIR) {
            using Cfg2 = Fused2Cfg<L, TX2, TY2>;
            e = occupancy(k_step_fused2<L, S, TX2, TY2, AB::MINB>, Cfg2::NTH, Cfg2::smem);
        } else {
            using Cfg1 = FusedCfg<L, TX2, TY2>;
            e = occupancy(k_step_fused<L, S, TX2, TY2>, Cfg1::NT, Cfg1::smem);
        }
        if (e != cudaSuccess) return e;
    } else {
        // the fewer resident blocks of the two forms
        auto ke = k_step_inplace<L, S, TX, TY, STEP_EVEN>;
        auto ko = k_step_inplace<L, S, TX, TY, STEP_ODD>;
        int pe = 0, po = 0;
        if ((e = cudaFuncSetAttribute(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem))) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(ko, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem))) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pe, ke, Cfg::NT, Cfg::smem)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&po, ko, Cfg::NT, Cfg::smem)) != cudaSuccess) return e;
        per_sm = pe < po ? pe : po;
        G->blocks_even = sms * (pe < 1 ? 1 : pe);       // the even form fills its own occupancy
    }
    per_sm = per_sm < 1 ? 1 : per_sm;
    const int slots = sms * per_sm;
    const int tx = inplace ? TX : TX2, ty = inplace ? TY : TY2;
    G->tiles_x = (P.nx + tx - 1) / tx;
    G->tiles_y = (L::D == 3) ? (P.ny + ty - 1) / ty : 1;
    G->ntiles = G->tiles_x * G->tiles_y;
    const int nm = (L::D == 3) ? P.nz : P.ny;
    // segments: the count that maximises the useful share of the slots'
    // work (items a multiple of the slots when that is possible, so every
    // persistent block gets equal work; each segment re-forms phi of two
    // extra planes); at least 2 planes each, so that a small grid is cut into
    // enough items to fill the GPU (a 128 x 128 grid: 128 items of 2 planes,
    // 4.5x faster per step than 16 items of 16 planes)
    int best = 1;
    double best_eff = -1.0;
    for (int nseg = 1; nseg <= nm; ++nseg) {
        const int seglen = (nm + nseg - 1) / nseg;
        if (seglen < 2 && nseg > 1) break;
        const long items = long(G->ntiles) * nseg;
        const long rounds = (items + slots - 1) / slots;
        const double work = double(nm + 2 * nseg);          // planes incl. the 2-plane prologue
        const double eff = (double(items) / double(rounds * slots)) * (double(nm) / work);
        if (eff > best_eff + 1e-9) { best_eff = eff; best = nseg; }
    }
    G->seglen = (nm + best - 1) / best;
    G->nseg = (nm + G->seglen - 1) / G->seglen;
    G->items = G->ntiles * G->nseg;
    *nblocks = G->items < slots ? G->items : slots;
    return cudaSuccess;
}

template <class L, class S>
cudaError_t Launch<L, S>::step_fused(const DevParams& P, const FusedGeom& G, int nblocks, const Buffers& b,
                                     cudaStream_t s)
{
    return step_timed(P, G, nblocks, b, s, nullptr, nullptr);
}

template <class L, class S>
cudaError_t Launch<L, S>::step_timed(const DevParams& P, const FusedGeom& G, int nblocks, const Buffers& b,
                                     cudaStream_t s, MarkFn markfn, void* mctx)
{
    auto mark = [&]() { return markfn ? markfn(mctx) : cudaSuccess; };
    constexpr int TX = InplaceTile<L>::TX, TY = InplaceTile<L>::TY;     // in-place forms
    using Cfg = FusedCfg<L, TX, TY>;
    const T* fA = static_cast<const T*>(b.fA);
    const T* gA = static_cast<const T*>(b.gA);
    T* fB = static_cast<T*>(b.inplace ? b.fA : b.fB);
    T* gB = static_cast<T*>(b.inplace ? b.gA : b.gB);
    const dim3 blk(TX, (L::D == 3) ? TY : 1);
    cudaError_t e;
    int par = 0;                                    // layout of the state after the step
    if (!b.inplace) {
        if ((e = mark()) != cudaSuccess) return e;  // no separate phi pass in the A/B step
        using AB = ABStep<L, S>;
        if constexpr (AB::PAIR) {
            using Cfg2 = Fused2Cfg<L, AB::TX, AB::TY>;
            const dim3 blk2(AB::TX / 2, (L::D == 3) ? AB::TY : 1);
            k_step_fused2<L, S, AB::TX, AB::TY, AB::MINB><<<nblocks, blk2, Cfg2::smem, s>>>(P, G, fA, gA, fB, gB);
        } else {
            using Cfg1 = FusedCfg<L, AB::TX, AB::TY>;
            const dim3 blk1(AB::TX, (L::D == 3) ? AB::TY : 1);
            k_step_fused<L, S, AB::TX, AB::TY><<<nblocks, blk1, Cfg1::smem, s>>>(P, G, fA, gA, fB, gB);
        }
    } else {
        // phi pre-pass into P.phis, then the even (natural -> swapped) or the
        // odd (swapped -> natural) in-place form
        k_phi_pre<L, S><<<dim3((P.nx + 127) / 128, P.ny, (L::D == 3) ? P.nz : 1), 128, 0, s>>>(P, gA, b.par, b.phi);
        if ((e = mark()) != cudaSuccess) return e;
        const int ne = G.blocks_even > 0 ? (G.blocks_even < G.items ? G.blocks_even : G.items) : nblocks;
        if (b.par == 0) k_step_inplace<L, S, TX, TY, STEP_EVEN><<<ne, blk, Cfg::smem, s>>>(P, G, fB, gB);
        else k_step_inplace<L, S, TX, TY, STEP_ODD><<<nblocks, blk, Cfg::smem, s>>>(P, G, fB, gB);
        par = b.par ^ 1;
    }
    if ((e = mark()) != cudaSuccess) return e;
    const int lastlo = (L::D == 2) ? P.bc[2] : P.bc[4];
    const int lasthi = (L::D == 2) ? P.bc[3] : P.bc[5];
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    if (lastlo == BC_INLET && lasthi == BC_OUTFLOW && !P.outlet_scheme) {
        // the jet: both face rules in one launch
        const unsigned nb = (2 * nface + 127) / 128;
        if (b.inplace) k_faces<L, S, true><<<nb, 128, 0, s>>>(P, fA, gA, fB, gB, par);
        else k_faces<L, S, false><<<nb, 128, 0, s>>>(P, fA, gA, fB, gB, par);
    } else {
        if (lastlo == BC_INLET) k_inlet<L, S><<<(nface + 127) / 128, 128, 0, s>>>(P, fB, gB, par);
        if (lasthi == BC_OUTFLOW) {
            if (P.outlet_scheme) k_outlet_speed<L, S><<<1, 256, 0, s>>>(P, fB, par);
            if (b.inplace) k_outlet<L, S, true><<<(nface + 127) / 128, 128, 0, s>>>(P, fA, gA, fB, gB, par);
            else k_outlet<L, S, false><<<(nface + 127) / 128, 128, 0, s>>>(P, fA, gA, fB, gB, par);
        }
    }
    if ((e = mark()) != cudaSuccess) return e;
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::save_outlet(const DevParams& P, const Buffers& b, cudaStream_t s)
{
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    k_save_outlet<L, S><<<(nface + 127) / 128, 128, 0, s>>>(P, static_cast<const T*>(b.fA), static_cast<const T*>(b.gA),
                                                           b.par);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::init(const DevParams& P, const float* phi, const float* u, const float* pstar, void* f,
                               void* g, cudaStream_t s)
{
    k_init<L, S><<<unsigned((P.N + 255) / 256), 256, 0, s>>>(P, phi, u, pstar, static_cast<T*>(f),
                                                             static_cast<T*>(g));
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::fields(const DevParams& P, const Buffers& b, float* ophi, float* ou, float* op,
                                 cudaStream_t s)
{
    const T* fA = static_cast<const T*>(b.fA);
    const T* gA = static_cast<const T*>(b.gA);
    k_phi<L, S, false><<<unsigned((P.N + 127) / 128), 128, 0, s>>>(P, gA, b.par, b.phi);
    dim3 grid((P.nx + 127) / 128, P.ny, (L::D == 3) ? P.nz : 1);
    k_fields<L, S><<<grid, 128, 0, s>>>(P, fA, gA, b.par, b.phi, ophi, ou, op);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::diag(const DevParams& P, const Buffers& b, double eps, DiagPartial* part, int nparts,
                               DiagPartial* res, cudaStream_t s)
{
    const T* fA = static_cast<const T*>(b.fA);
    const T* gA = static_cast<const T*>(b.gA);
    k_phi<L, S, false><<<unsigned((P.N + 127) / 128), 128, 0, s>>>(P, gA, b.par, b.phi);
    k_diag<L, S, false><<<nparts, 256, 0, s>>>(P, fA, gA, b.par, b.phi, eps, part);
    k_diag_final<L><<<1, 32, 0, s>>>(part, nparts, res);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::diag_planar(const DevParams& P, const Buffers& b, double eps, DiagPartial* part,
                                      int nparts, DiagPartial* res, cudaStream_t s)
{
    const T* fA = static_cast<const T*>(b.fA);
    const T* gA = static_cast<const T*>(b.gA);
    k_phi<L, S, true><<<unsigned((P.N + 127) / 128), 128, 0, s>>>(P, gA, 0, b.phi);
    k_diag<L, S, true><<<nparts, 256, 0, s>>>(P, fA, gA, 0, b.phi, eps, part);
    k_diag_final<L><<<1, 32, 0, s>>>(part, nparts, res);
    return cudaGetLastError();
}

// Populations a0 .. a1-1 of one set of the state (par: swapped) into float32
// planes out[(a - a0) N + node]; gset: the set is g (else f).
template <class L, class S>
__global__ void k_unpack(const __grid_constant__ DevParams P, const typename S::T* __restrict__ src, int gset,
                         int par, int a0, int a1, float* __restrict__ out)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = int(i % P.nx), y = int((i / P.nx) % P.ny), z = int(i / (int64_t(P.nx) * P.ny));
    for (int a = a0; a < a1; ++a) {
        const uint32_t e = post_el<L>(P, x, y, z, a, par);
        out[(a - a0) * P.N + i] = gset ? S::g(src[e], L::w(a)) : S::f(src[e], L::w(a), fref<S>(P, march<L>(y, z)), P);
    }
}

// float32 planes in[(a - a0) N + node] into populations a0 .. a1-1 of one set
// of the state, natural layout; gset: the set is g (else f).
template <class L, class S>
__global__ void k_pack(const __grid_constant__ DevParams P, const float* __restrict__ in, int gset, int a0, int a1,
                       typename S::T* __restrict__ dst)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int x = int(i % P.nx), y = int((i / P.nx) % P.ny), z = int(i / (int64_t(P.nx) * P.ny));
    const uint32_t e = pel<L>(pnode(P, x, y, z));
    const float r = gset ? 0.0f : fref<S>(P, march<L>(y, z));
    for (int a = a0; a < a1; ++a) {
        const float v = in[(a - a0) * P.N + i];
        dst[e + 32 * a] = gset ? S::eg(v, L::w(a)) : S::ef(v, L::w(a), r, P);
    }
}

template <class L, class S>
cudaError_t Launch<L, S>::unpack(const DevParams& P, const Buffers& b, int gset, int a0, int a1, float* out,
                                 cudaStream_t s)
{
    k_unpack<L, S><<<unsigned((P.N + 255) / 256), 256, 0, s>>>(P, static_cast<const T*>(gset ? b.gA : b.fA), gset,
                                                               b.par, a0, a1, out);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::pack(const DevParams& P, const float* in, int gset, int a0, int a1, void* dst,
                               cudaStream_t s)
{
    k_pack<L, S><<<unsigned((P.N + 255) / 256), 256, 0, s>>>(P, in, gset, a0, a1, static_cast<T*>(dst));
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::inlet_profile(const DevParams& P, double cx, double cy, double R, double W, double uj,
                                        float* phi_in, float* u_in, cudaStream_t s)
{
    const int nface = (L::D == 2) ? P.nx : P.nx * P.ny;
    k_inlet_profile<L><<<(nface + 127) / 128, 128, 0, s>>>(nface, P.nx, cx, cy, R, W, uj, phi_in, u_in);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::phi(const DevParams& P, const Buffers& b, cudaStream_t s)
{
    k_phi<L, S, false><<<unsigned((P.N + 127) / 128), 128, 0, s>>>(P, static_cast<const T*>(b.gA), b.par, b.phi);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::plane_ref(const DevParams& P, const float* X, float scale, float* ref, cudaStream_t s)
{
    const int nm = (L::D == 3) ? P.nz : P.ny;
    if (!X) return cudaMemsetAsync(ref, 0, sizeof(float) * size_t(nm), s);
    k_plane_ref<L><<<unsigned(nm), 256, 0, s>>>(P, X, scale, ref);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::advect(const DevParams& P, const Buffers& b, const float* uf, float scale, cudaStream_t s)
{
    k_phi<L, S, false><<<unsigned((P.N + 127) / 128), 128, 0, s>>>(P, static_cast<const T*>(b.gA), 0, b.phi);
    k_advect<L, S><<<unsigned((P.N + 127) / 128), 128, 0, s>>>(P, b.phi, uf, scale, static_cast<const T*>(b.gA),
                                                               static_cast<T*>(b.gB));
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::collide_cells(const DevParams& P, int64_t n, const float* f, const float* g,
                                        const float* phin, float* fs, float* gs, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_collide_cells<L><<<unsigned((n + 127) / 128), 128, 0, s>>>(P, n, f, g, phin, fs, gs, out);
    return cudaGetLastError();
}

// Launcher of the batched step for one tile shape.
template <class L, class S, int TX, int TY>
struct BatchLaunch {
    using T = typename S::T;
    static constexpr int NT = TX * ((L::D == 3) ? TY : 1);
    // sets the kernel's shared-memory limit; *per_sm = resident blocks per SM
    static cudaError_t setup(int* per_sm);
    static cudaError_t step(const BatchCase* cases, const int2* items, int nitems, int* counter, int nblocks,
                            const void* fA, const void* gA, void* fB, void* gB, cudaStream_t s);
};

template <class L, class S, int TX, int TY>
cudaError_t BatchLaunch<L, S, TX, TY>::setup(int* per_sm)
{
    using Cfg = FusedCfg<L, TX, TY>;
    auto kern = k_step_batch<L, S, TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg::smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, NT, Cfg::smem);
}

template <class L, class S, int TX, int TY>
cudaError_t BatchLaunch<L, S, TX, TY>::step(const BatchCase* cases, const int2* items, int nitems, int* counter,
                                            int nblocks, const void* fA, const void* gA, void* fB, void* gB,
                                            cudaStream_t s)
{
    using Cfg = FusedCfg<L, TX, TY>;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_step_batch<L, S, TX, TY><<<nblocks, dim3(TX, (L::D == 3) ? TY : 1), Cfg::smem, s>>>(
        cases, items, nitems, counter, static_cast<const T*>(fA), static_cast<const T*>(gA), static_cast<T*>(fB),
        static_cast<T*>(gB));
    return cudaGetLastError();
}

}  // namespace lbm
