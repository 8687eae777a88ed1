// Device kernels of the GB300 library for the 3D DDF-MRT porous-convection model
// (Liu & He, arXiv:1611.03329).
//
// Storage: FP32 deviations f'_i = f_i - w_i rho0 and g'_i = g_i - omega_i sigma T0, planes of
// sq floats per population, f planes 0..18 then g planes 19..25, x-fastest sites.  The
// moment-space equilibria are affine in rho and in sigma T, so the collision runs on the
// deviations directly (rho is replaced by rho' = rho - rho0, sigma T by sigma (T - T0)).
//
// One thread updates one site: pull 26 populations (Eqs. 10, 35 with the wall rules),
// collide in moment space with the sparse integer M of Eq. A2 and N of Eq. 36 unrolled in
// registers, push the back-transform through M^-1 = M^T diag(1/|M_k|^2) (the rows of Eq. A2
// are orthogonal) and N^-1 of Eq. 43, and store 26 populations.  Threads are laid out as a
// 3D grid (x fastest, one z-plane per grid slice) so that no index division is needed; a
// warp whose 32 sites are all interior takes unconditional loads, any other warp takes the
// predicated boundary path.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <utility>
#include <type_traits>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

// ---- lattice constants -------------------------------------------------------------------
// D3Q19 velocity components, Eq. 19.
__host__ __device__ constexpr int ex19(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int ey19(int i) {
    return (i == 3 || i == 7 || i == 8 || i == 15 || i == 17)    ? 1
           : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int ez19(int i) {
    return (i == 5 || i == 11 || i == 12 || i == 15 || i == 16)  ? 1
           : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int opp19(int i) {
    return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : 7 + 4 * ((i - 7) / 4) + 3 - (i - 7) % 4);
}
// Weights stated under Eq. 24.
__host__ __device__ constexpr float w19(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
// Slot of the outflow history for the five D3Q19 velocities with e_x = -1.
__host__ __device__ constexpr int slot19(int i) {
    return i == 2 ? 0 : i == 8 ? 1 : i == 10 ? 2 : i == 12 ? 3 : i == 14 ? 4 : -1;
}
// D3Q7 velocity components (first seven columns of Eq. 12).
__host__ __device__ constexpr int ex7(int i) { return i == 1 ? 1 : i == 2 ? -1 : 0; }
__host__ __device__ constexpr int ey7(int i) { return i == 3 ? 1 : i == 4 ? -1 : 0; }
__host__ __device__ constexpr int ez7(int i) { return i == 5 ? 1 : i == 6 ? -1 : 0; }
__host__ __device__ constexpr int opp7(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Flow lattices as traits of the site kernels: D3Q19 (Eq. 19, the default) and D3Q15
// (Eq. 12).  Both put the velocities with e_x = -1 at 2, 8, 10, 12, 14 (the outflow slots).
struct D3Q19 {
    static constexpr int kQ = 19;
    __host__ __device__ static constexpr int ex(int i) { return ex19(i); }
    __host__ __device__ static constexpr int ey(int i) { return ey19(i); }
    __host__ __device__ static constexpr int ez(int i) { return ez19(i); }
    __host__ __device__ static constexpr int opp(int i) { return opp19(i); }
    __host__ __device__ static constexpr float w(int i) { return w19(i); }
    __host__ __device__ static constexpr double wd(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int slot(int i) { return slot19(i); }
};
struct D3Q15 {
    static constexpr int kQ = 15;
    __host__ __device__ static constexpr int ex(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
               : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                      : 0;
    }
    __host__ __device__ static constexpr int ey(int i) {
        return (i == 3 || i == 7 || i == 8 || i == 11 || i == 12)    ? 1
               : (i == 4 || i == 9 || i == 10 || i == 13 || i == 14) ? -1
                                                                      : 0;
    }
    __host__ __device__ static constexpr int ez(int i) {
        return (i == 5 || i == 7 || i == 8 || i == 9 || i == 10)     ? 1
               : (i == 6 || i == 11 || i == 12 || i == 13 || i == 14) ? -1
                                                                       : 0;
    }
    __host__ __device__ static constexpr int opp(int i) {
        return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : 21 - i);
    }
    // weights stated under Eq. 18
    __host__ __device__ static constexpr float w(int i) {
        return i == 0 ? 2.0f / 9.0f : (i <= 6 ? 1.0f / 9.0f : 1.0f / 72.0f);
    }
    __host__ __device__ static constexpr double wd(int i) {
        return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
    __host__ __device__ static constexpr int slot(int i) { return slot19(i); }
};
template <class L>
constexpr bool lattice_consistent() {
    for (int i = 0; i < L::kQ; ++i) {
        const int o = L::opp(i);
        if (L::opp(o) != i || L::ex(o) != -L::ex(i) || L::ey(o) != -L::ey(i) ||
            L::ez(o) != -L::ez(i))
            return false;
        if ((L::ex(i) == -1) != (L::slot(i) >= 0)) return false;
    }
    return true;
}
static_assert(lattice_consistent<D3Q19>() && lattice_consistent<D3Q15>(), "lattice tables");

static_assert(opp19(7) == 10 && opp19(8) == 9 && opp19(12) == 13 && opp19(16) == 17, "opp19");
static_assert(ex19(opp19(13)) == -ex19(13) && ez19(opp19(13)) == -ez19(13), "opp19 sign");

// ---- population storage ------------------------------------------------------------------
// FP32 planes hold the deviation f - w_i rho0 (g - omega_i sigma T0) itself.  The 16-bit
// formats hold kFlowUnit (f - w_i rho0) for the D3Q19 planes (a power of two, so the loads
// and stores are conversions only and the flow collision runs in these units; the factor
// keeps the smallest deviations out of the FP16 subnormal range) and (g - omega_i sigma T_x) /
// omega_i for the D3Q7 planes, against the site's own temperature T_x kept in an FP32 plane
// (ldg_dev).  Arithmetic is FP32 in every case; 16-bit values are rounded to nearest on store.
// kStrided: plane q is addressed as plane 0 + q * sq (the planes of a copy are contiguous)
// instead of through its own pointer.  Fewer pointer loads from the parameter block (which go
// through the address-divergence pipe) for more integer adds; the 16-bit step measured 13 %
// faster, FP32 the same, so only the 16-bit formats use it.
// kOff32: plane q at element offset Planes::off_in[q] / off_out[q] from one base pointer per
// side, the offset and the site index added in 32 bits and widened once (two integer
// instructions per access, no pointer read from the parameter block); used by the hot
// kernels when every offset of a copy fits an int (KParams::off32).
struct StoreF32 {
    using T = float;
    static constexpr bool kScaled = false;
    static constexpr bool kStrided = false;
    static constexpr bool kOff32 = false;
    static __device__ __forceinline__ float ld(const T* q) { return __ldg(q); }
    static __device__ __forceinline__ void st(T* q, float v) { *q = v; }
};
struct StoreF16 {
    using T = __half;
    static constexpr bool kScaled = true;
    static constexpr bool kStrided = true;
    static constexpr bool kOff32 = false;
    static __device__ __forceinline__ float ld(const T* q) { return __half2float(__ldg(q)); }
    static __device__ __forceinline__ void st(T* q, float v) { *q = __float2half_rn(v); }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    static constexpr bool kScaled = true;
    static constexpr bool kStrided = true;
    static constexpr bool kOff32 = false;
    static __device__ __forceinline__ float ld(const T* q) { return __bfloat162float(__ldg(q)); }
    static __device__ __forceinline__ void st(T* q, float v) { *q = __float2bfloat16_rn(v); }
};
// A storage format addressed by 32-bit offsets (see kOff32 above).
template <class B>
struct Off32 : B {
    static constexpr bool kOff32 = true;
};
using StoreF32o = Off32<StoreF32>;
using StoreF16o = Off32<StoreF16>;
using StoreBF16o = Off32<StoreBF16>;

// Optional bounds checks (compile with -DLBM_BOUNDS_CHECK): every site index of a population,
// temperature-plane, porosity or outflow-history access is checked; an index out of range is
// recorded (the first one met, in g_bounds_bad) and replaced by 0, so the kernel goes on
// without touching memory outside its buffers.  Without the macro the check is the identity.
#ifdef LBM_BOUNDS_CHECK
__device__ unsigned long long g_bounds_bad;  // 0, or 1 + the first out-of-range index met
__device__ __forceinline__ int chk(int i, long long n) {
    if ((unsigned long long)(long long)i >= (unsigned long long)n) {
        atomicCAS(&g_bounds_bad, 0ull, 1ull + (unsigned long long)(unsigned)i);
        return 0;
    }
    return i;
}
#else
__device__ __forceinline__ int chk(int i, long long) { return i; }
#endif

// Start of plane q of the planes being read / written.
template <class S>
__device__ __forceinline__ const typename S::T* plane_in(const Planes& pl, const KParams& p, int q) {
    if constexpr (S::kStrided) return static_cast<const typename S::T*>(pl.in[0]) + q * p.sq;
    else return static_cast<const typename S::T*>(pl.in[q]);
}
template <class S>
__device__ __forceinline__ typename S::T* plane_out(const Planes& pl, const KParams& p, int q) {
    if constexpr (S::kStrided) return static_cast<typename S::T*>(pl.out[0]) + q * p.sq;
    else return static_cast<typename S::T*>(pl.out[q]);
}
// Element idx of plane q of the planes being read / written; the `either` form takes plane J
// instead of I when `other` is set.
template <class S>
__device__ __forceinline__ const typename S::T* at_in(const Planes& pl, const KParams& p, int q,
                                                      int idx) {
    idx = chk(idx, p.ns);
    if constexpr (S::kOff32)
        return static_cast<const typename S::T*>(pl.base_in) + (unsigned)(pl.off_in[q] + idx);
    else
        return plane_in<S>(pl, p, q) + idx;
}
template <class S>
__device__ __forceinline__ typename S::T* at_out(const Planes& pl, const KParams& p, int q, int idx) {
    idx = chk(idx, p.ns);
    if constexpr (S::kOff32)
        return static_cast<typename S::T*>(pl.base_out) + (unsigned)(pl.off_out[q] + idx);
    else
        return plane_out<S>(pl, p, q) + idx;
}
// Element idx + d of plane q of the planes being read, addressed from element idx: elements
// next to each other share one address computation.  The bounds-checked build checks idx + d.
template <class S>
__device__ __forceinline__ const typename S::T* at_in_rel(const Planes& pl, const KParams& p, int q,
                                                          int idx, int d) {
#ifdef LBM_BOUNDS_CHECK
    return at_in<S>(pl, p, q, idx + d);
#else
    return at_in<S>(pl, p, q, idx) + d;
#endif
}
template <class S>
__device__ __forceinline__ const typename S::T* at_in_either(const Planes& pl, const KParams& p,
                                                             int I, int J, bool other, int idx) {
    idx = chk(idx, p.ns);
    if constexpr (S::kOff32)
        return static_cast<const typename S::T*>(pl.base_in) +
               (unsigned)((other ? pl.off_in[J] : pl.off_in[I]) + idx);
    else
        return (other ? plane_in<S>(pl, p, J) : plane_in<S>(pl, p, I)) + idx;
}
// Deviation of plane q at site index idx of the planes being read / written, in the flow unit
// of the format (kFlowUnit for a 16-bit D3Q19 plane): decoding and encoding are conversions
// only.  D3Q7 planes go through these only in FP32 (16-bit: ldg_dev / stg_dev).
template <class S>
__device__ __forceinline__ float ldp(const Planes& pl, const KParams& p, int q, int idx) {
    return S::ld(at_in<S>(pl, p, q, idx));
}
template <class S>
__device__ __forceinline__ void stp(const Planes& pl, const KParams& p, int q, int idx, float v) {
    S::st(at_out<S>(pl, p, q, idx), v);
}
// D3Q7 population i at site idx as the deviation g_i - omega_i sigma T0.  The 16-bit formats
// store (g_i - omega_i sigma T_x) / omega_i against the site's own temperature T_x, whose
// deviation T_x - T0 sits in an FP32 plane (tin / tout): thermal populations are then of the
// order of T u / c_sT^2 instead of T - T0, and keep their precision.
template <class S>
__device__ __forceinline__ float ldg_dev(const Planes& pl, const KParams& p, int i, int idx) {
    if constexpr (!S::kScaled) {
        return ldp<S>(pl, p, kQ + i, idx);
    } else {
        // explicit roundings (no contraction left to the compiler): the staged-load kernel
        // repeats this arithmetic and must give the same bits
        const float sc = i == 0 ? p.om0 : p.om1;
        return __fmul_rn(sc, __fmaf_rn(p.sigma, __ldg(pl.tin + chk(idx, p.ns)),
                                       S::ld(at_in<S>(pl, p, kQ + i, idx))));
    }
}
// Stores post-collision g' (deviation from omega_i sigma T0) of a site whose temperature
// deviation is dT.
template <class S>
__device__ __forceinline__ void stg_dev(const Planes& pl, const KParams& p, int i, int idx, float v,
                                        float dT) {
    if constexpr (!S::kScaled) {
        stp<S>(pl, p, kQ + i, idx, v);
    } else {
        const float isc = i == 0 ? p.iom0 : p.iom1;
        S::st(at_out<S>(pl, p, kQ + i, idx), __fmaf_rn(v, isc, -__fmul_rn(p.sigma, dT)));
    }
}

// ---- site and neighbourhood ----------------------------------------------------------------
// A site with the offsets (in sites) of its six axis neighbours' sources and the faces that
// a pull would cross.  For a velocity with component +1 along an axis the source lies at -1
// (offset *m); with -1 at +1 (offset *p).  Periodic faces wrap the offset; a non-periodic
// face sets its bit in `cross` (bits: x-low, x-high, y-low, y-high, z-low, z-high).
struct Nbr {
    int x, y, z, s;
    int xm, xp, ym, yp, zm, zp;
    unsigned cross;
};

__device__ __forceinline__ Nbr neighbourhood(const KParams& p, int x, int y, int z) {
    Nbr n;
    n.x = x;
    n.y = y;
    n.z = z;
    const int nxy = p.nx * p.ny;
    n.s = x + p.nx * (y + p.ny * z);
    n.cross = 0u;
    n.xm = -1;
    n.xp = 1;
    n.ym = -p.nx;
    n.yp = p.nx;
    n.zm = -nxy;
    n.zp = nxy;
    if (x == 0) { if (p.per_mask & 1u) n.xm = p.nx - 1; else { n.xm = 0; n.cross |= 1u; } }
    if (x == p.nx - 1) { if (p.per_mask & 2u) n.xp = 1 - p.nx; else { n.xp = 0; n.cross |= 2u; } }
    if (y == 0) { if (p.per_mask & 4u) n.ym = p.nx * (p.ny - 1); else { n.ym = 0; n.cross |= 4u; } }
    if (y == p.ny - 1) { if (p.per_mask & 8u) n.yp = -p.nx * (p.ny - 1); else { n.yp = 0; n.cross |= 8u; } }
    if (z == 0) { if (p.per_mask & 16u) n.zm = nxy * (p.nz - 1); else { n.zm = 0; n.cross |= 16u; } }
    if (z == p.nz - 1) { if (p.per_mask & 32u) n.zp = -nxy * (p.nz - 1); else { n.zp = 0; n.cross |= 32u; } }
    return n;
}

// Source offset along one axis for velocity component e: +1 pulls from -1 and vice versa.
__device__ __forceinline__ int axis_off(int e, int m, int p_) { return e == 1 ? m : (e == -1 ? p_ : 0); }
__device__ __forceinline__ unsigned axis_cross(int e, unsigned cr, unsigned lo, unsigned hi) {
    return e == 1 ? (cr & lo) : (e == -1 ? (cr & hi) : 0u);
}

// ---- arithmetic on one site or on an x-adjacent pair of sites --------------------------------
// The collision is written once over a lane type: L1 carries one site (FP32 instructions), L2
// two sites (the paired FP32 instructions FADD2, FMUL2, FFMA2 of sm_100).  Every operation
// rounds explicitly -- nothing is left to the compiler to contract into an FMA -- so a site
// gives the same bits updated alone or paired, in whatever kernel inlines the update.
struct L1 {
    float v;
};
struct L2 {
    float2 v;
};
__device__ __forceinline__ L1 operator+(L1 a, L1 b) { return {__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ L1 operator-(L1 a, L1 b) { return {__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ L1 operator*(L1 a, L1 b) { return {__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ L1 operator-(L1 a) { return {-a.v}; }
__device__ __forceinline__ L1 fma(L1 a, L1 b, L1 c) { return {__fmaf_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ L2 operator+(L2 a, L2 b) { return {__fadd2_rn(a.v, b.v)}; }
// a - b as b * (-1) + a: one rounding of the exact difference, as __fsub_rn
__device__ __forceinline__ L2 operator-(L2 a, L2 b) {
    return {__ffma2_rn(b.v, make_float2(-1.0f, -1.0f), a.v)};
}
__device__ __forceinline__ L2 operator*(L2 a, L2 b) { return {__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ L2 operator-(L2 a) { return {make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ L2 fma(L2 a, L2 b, L2 c) { return {__ffma2_rn(a.v, b.v, c.v)}; }
// a constant on every lane
template <class V> __device__ __forceinline__ V K(float c);
template <> __device__ __forceinline__ L1 K<L1>(float c) { return {c}; }
template <> __device__ __forceinline__ L2 K<L2>(float c) { return {make_float2(c, c)}; }
// lane-wise application of a scalar function (the special-function steps)
template <class F> __device__ __forceinline__ L1 lanes(L1 a, F fn) { return {fn(a.v)}; }
template <class F> __device__ __forceinline__ L2 lanes(L2 a, F fn) {
    return {make_float2(fn(a.v.x), fn(a.v.y))};
}
template <class F> __device__ __forceinline__ L1 lanes(L1 a, L1 b, F fn) { return {fn(a.v, b.v)}; }
template <class F> __device__ __forceinline__ L2 lanes(L2 a, L2 b, F fn) {
    return {make_float2(fn(a.v.x, b.v.x), fn(a.v.y, b.v.y))};
}

// sqrt of a non-negative value through the hardware reciprocal square root (exact zero kept).
__device__ __forceinline__ float sqrt_nonneg(float v) {
    return v > 0.0f ? __fmul_rn(v, rsqrtf(v)) : 0.0f;
}

template <class V>
struct MediumT {
    V phi, inv_phi, l0, l1, c_darcy, c_forch, zeta_alpha;
};
using Medium = MediumT<L1>;

// Eq. 4 / Eq. 28 coefficients at a site; Eq. 6 (Kozeny-Carman K, Ergun F_phi) for a field.
template <bool HET>
__device__ __forceinline__ Medium medium_at(const KParams& p, int s) {
    Medium m;
    if (!HET) {
        m.phi = {p.phi};
        m.inv_phi = {p.inv_phi};
        m.l0 = {p.l0};
        m.l1 = {p.l1};
        m.c_darcy = {p.c_darcy};
        m.c_forch = {p.c_forch};
        m.zeta_alpha = {p.zeta_alpha};
    } else {
        const float ph = __ldg(p.phi_field + chk(s, p.ns));
        const float ph3 = __fmul_rn(__fmul_rn(ph, ph), ph);
        const float omp = __fsub_rn(1.0f, ph);
        const float Fp = p.F_phi < 0.0f ? __fmul_rn(1.75f, rsqrtf(__fmul_rn(150.0f, ph3))) : p.F_phi;
        const float inv_sqrtK = p.kinf ? 0.0f : __fmul_rn(omp, rsqrtf(__fmul_rn(p.cK, ph3)));
        m.phi = {ph};
        m.inv_phi = {__fdividef(1.0f, ph)};
        const float cd = __fmul_rn(__fmul_rn(__fmul_rn(ph, p.nu), inv_sqrtK), inv_sqrtK);  // phi nu / K
        const float cf = __fmul_rn(__fmul_rn(ph, Fp), inv_sqrtK);  // phi F_phi / sqrt(K)
        m.c_darcy = {cd};
        m.c_forch = {cf};
        m.l0 = {__fmul_rn(0.5f, __fmaf_rn(0.5f, cd, 1.0f))};
        m.l1 = {__fmul_rn(0.5f, cf)};
        m.zeta_alpha = {p.hetero_alpha
                            ? __fdividef(1.0f, __fmaf_rn(__fmaf_rn(ph, p.alpha_f,
                                                                   __fmul_rn(omp, p.alpha_m)),
                                                         p.inv_sig_csT2, 0.5f))
                            : p.zeta_alpha};
    }
    return m;
}
// The medium of the two sites of a pair (each computed as medium_at computes it).
template <bool HET>
__device__ __forceinline__ MediumT<L2> medium_pair(const KParams& p, int sa) {
    const Medium a = medium_at<HET>(p, sa), b = medium_at<HET>(p, sa + 1);
    auto pk = [](L1 x, L1 y) { return L2{make_float2(x.v, y.v)}; };
    return {pk(a.phi, b.phi), pk(a.inv_phi, b.inv_phi), pk(a.l0, b.l0), pk(a.l1, b.l1),
            pk(a.c_darcy, b.c_darcy), pk(a.c_forch, b.c_forch), pk(a.zeta_alpha, b.zeta_alpha)};
}

// ---- streaming with boundary rules ------------------------------------------------------------
// The three value rules of a pull that crosses a face, each written with explicit roundings so
// that every kernel that inlines them (plain, batched, AA, staged) computes the same bits.
// Moving wall / velocity inlet (halfway bounce-back with the wall's momentum):
// f_I = f*_opp(I)(x) + 2 w_I rho0 (e_I . u_w) / c_s^2, u_w the velocity of `face`.
template <class L, int I>
__device__ __forceinline__ float bounce_moving(const KParams& p, int face, float bb) {
    // e_I has components in {-1, 0, 1}: the products are exact, the two sums round in order
    const float eu = __fadd_rn(__fadd_rn((float)L::ex(I) * p.face_u[face][0],
                                         (float)L::ey(I) * p.face_u[face][1]),
                               (float)L::ez(I) * p.face_u[face][2]);
    return __fmaf_rn(__fmul_rn(6.0f * L::w(I), p.frho0), eu, bb);
}
// The same for a pull of I that crosses the velocity faces vm (non-zero): the lowest-numbered
// one applies.  The candidate faces are those along I's non-zero components, known at compile
// time, so the face velocity is picked with selects of parameter values instead of an
// indexed read of the parameter block.
template <class L, int I>
__device__ __forceinline__ float bounce_moving_on(const KParams& p, unsigned vm, float bb) {
    constexpr int ex = L::ex(I), ey = L::ey(I), ez = L::ez(I);
    constexpr int fx = ex == 1 ? 0 : 1, fy = ey == 1 ? 2 : 3, fz = ez == 1 ? 4 : 5;
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
    bool found = false;
    if constexpr (ex != 0) {
        if (vm & (1u << fx)) {
            u0 = p.face_u[fx][0]; u1 = p.face_u[fx][1]; u2 = p.face_u[fx][2];
            found = true;
        }
    }
    if constexpr (ey != 0) {
        if (!found && (vm & (1u << fy))) {
            u0 = p.face_u[fy][0]; u1 = p.face_u[fy][1]; u2 = p.face_u[fy][2];
            found = true;
        }
    }
    if constexpr (ez != 0) {
        if (!found) { u0 = p.face_u[fz][0]; u1 = p.face_u[fz][1]; u2 = p.face_u[fz][2]; }
    }
    const float eu = __fadd_rn(__fadd_rn((float)ex * u0, (float)ey * u1), (float)ez * u2);
    return __fmaf_rn(__fmul_rn(6.0f * L::w(I), p.frho0), eu, bb);
}
// Face a D3Q7 velocity crosses (each has one non-zero component): x-low, x-high, y-low, ...
constexpr int face7(int i) {
    return ex7(i) == 1 ? 0 : ex7(i) == -1 ? 1 : ey7(i) == 1 ? 2 : ey7(i) == -1 ? 3 : ez7(i) == 1 ? 4 : 5;
}
// Convective outflow: p(N-1, t+1) = (p(N-1, t) + U p(N-2, t+1)) / (1 + U) = a old + b inner.
__device__ __forceinline__ float outflow_blend(const KParams& p, float old, float inner) {
    return __fmaf_rn(p.out_a, old, __fmul_rn(p.out_b, inner));
}
// Pressure anchor of the outlet: the populations set by the outflow rule (`via`) are shifted by
// w_i (rho0 - rho) / sum(w_i) so that the outlet density is rho0; f holds deviations, so
// rho0 - rho = -sum f.  With all five entering velocities set by the rule, sum(w_i) = 1/6 on
// both lattices and the shift is w_i (-6 rho).
template <class L>
__device__ __forceinline__ void outflow_anchor(float* f, const bool* via) {
    float rho = 0.0f, wsum = 0.0f;
    int n = 0;
#pragma unroll
    for (int i = 0; i < L::kQ; ++i) {
        rho += f[i];
        if (via[i]) {
            wsum += L::w(i);
            ++n;
        }
    }
    if (n == 0) return;
    const float corr = n == 5 ? __fmul_rn(-6.0f, rho) : -rho / wsum;
#pragma unroll
    for (int i = 0; i < L::kQ; ++i)
        if (via[i]) f[i] = __fmaf_rn(L::w(i), corr, f[i]);
}

// Pull of f_I at site n: the post-collision population at x - e_I, or the wall rule when that
// source lies outside (a no-slip wall wins over a velocity face, which wins over the outflow).
template <class L, int I, bool OUTF, class S>
__device__ __forceinline__ float pull_f(const Planes& pl, const KParams& p, const Nbr& n,
                                        bool* via) {
    constexpr int ex = L::ex(I), ey = L::ey(I), ez = L::ez(I);
    const int oyz = axis_off(ey, n.ym, n.yp) + axis_off(ez, n.zm, n.zp);
    const unsigned cyz = axis_cross(ey, n.cross, 4u, 8u) | axis_cross(ez, n.cross, 16u, 32u);
    const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | cyz;
    if (cr == 0u) return ldp<S>(pl, p, I, n.s + axis_off(ex, n.xm, n.xp) + oyz);
    const float bb = ldp<S>(pl, p, L::opp(I), n.s);
    if (cr & p.wall_mask) return bb;
    unsigned vm = cr & p.vel_mask;
    if (vm) return bounce_moving_on<L, I>(p, vm, bb);
    if constexpr (OUTF && ex == -1) {
        // convective outflow with p(N-2, t+1) pulled at the inner neighbour: the source of
        // x - 1 along -x is x itself, at the same y/z offsets (a y/z face crossed here is a
        // wall or velocity face, taken above)
        *via = true;
        const float inner = ldp<S>(pl, p, I, n.s + oyz);
        const float old = __ldg(pl.hin + L::slot(I) * p.nyz + chk(n.y + p.ny * n.z, p.nyz));
        return outflow_blend(p, old, inner);
    }
    return bb;  // not reached for validated boundary sets
}

template <int I, bool OUTF, class S>
__device__ __forceinline__ float pull_g(const Planes& pl, const KParams& p, const Nbr& n) {
    constexpr int ex = ex7(I), ey = ey7(I), ez = ez7(I);
    const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                        axis_cross(ez, n.cross, 16u, 32u);
    if (cr == 0u)
        return ldg_dev<S>(pl, p, I, n.s + axis_off(ex, n.xm, n.xp) + axis_off(ey, n.ym, n.yp) +
                     axis_off(ez, n.zm, n.zp));
    constexpr int face = face7(I);  // a D3Q7 velocity crosses one face at most
    const int kind = p.heat_kind[face];
    if constexpr (OUTF && ex == -1) {
        if (kind == 3) {  // g_I(N-2, t+1) = g*_I(N-1, t)
            const float inner = ldg_dev<S>(pl, p, I, n.s);
            return outflow_blend(p, __ldg(pl.hin + 5 * p.nyz + chk(n.y + p.ny * n.z, p.nyz)), inner);
        }
    }
    const float bb = ldg_dev<S>(pl, p, opp7(I), n.s);
    if (kind == 2) return -bb + p.heat_abb[face];  // Dirichlet: anti-bounce-back
    return bb;                                      // adiabatic: bounce-back
}

template <class L, bool OUTF, class S, int... I>
__device__ __forceinline__ void gather_f_bc(float* f, bool* via, const Planes& pl,
                                            const KParams& p, const Nbr& n,
                                            std::integer_sequence<int, I...>) {
    ((f[I] = pull_f<L, I, OUTF, S>(pl, p, n, &via[I])), ...);
}

template <bool OUTF, class S, int... I>
__device__ __forceinline__ void gather_g_bc(float* g, const Planes& pl, const KParams& p,
                                            const Nbr& n, std::integer_sequence<int, I...>) {
    ((g[I] = pull_g<I, OUTF, S>(pl, p, n)), ...);
}

// Predicated pull of all populations (any site), with the outflow's pressure anchor.  Used
// where a site is gathered on its own (macroscopic fields, node walls, AA local steps).
template <bool OUTF, class S, class L = D3Q19>
__device__ __forceinline__ void gather_general(const Planes& pl, const KParams& p, const Nbr& n,
                                               float* f, float* g) {
    bool via[L::kQ];
#pragma unroll
    for (int i = 0; i < L::kQ; ++i) via[i] = false;
    gather_f_bc<L, OUTF, S>(f, via, pl, p, n, std::make_integer_sequence<int, L::kQ>{});
    gather_g_bc<OUTF, S>(g, pl, p, n, std::make_integer_sequence<int, kQT>{});
    if (OUTF && n.x == p.nx - 1) outflow_anchor<L>(f, via);
}

// The x-face rule after loads that ignored it (the staged-tile path of the TMA kernel): a lane
// on a non-periodic x face (cxm: x-low, cxp: x-high) replaces the populations that cross it.
// `lanes` names the lanes that call it together; oym, oyp, ozm, ozp are the site offsets of
// the pull sources of velocities with e_y = +1, -1 and e_z = +1, -1.
template <bool OUTF, class S, class L, int... I>
__device__ __forceinline__ void x_face_f(const Planes& pl, const KParams& p, int s, bool cxm,
                                         bool cxp, bool out, int oym, int oyp, int ozm, int ozp,
                                         int yz, float* f, bool* via,
                                         std::integer_sequence<int, I...>) {
    (([&] {
         if constexpr (L::ex(I) == 1) {
             if (cxm) {
                 const float bb = ldp<S>(pl, p, L::opp(I), s);
                 f[I] = ((p.vel_mask & 1u) && !(p.wall_mask & 1u)) ? bounce_moving<L, I>(p, 0, bb) : bb;
             }
         } else if constexpr (L::ex(I) == -1) {
             if (cxp) {
                 if (out) {
                     const float inner = ldp<S>(pl, p, I, s + axis_off(L::ey(I), oym, oyp) +
                                                              axis_off(L::ez(I), ozm, ozp));
                     f[I] = outflow_blend(p, __ldg(pl.hin + L::slot(I) * p.nyz + chk(yz, p.nyz)), inner);
                     via[I] = true;
                 } else {
                     const float bb = ldp<S>(pl, p, L::opp(I), s);
                     f[I] = ((p.vel_mask & 2u) && !(p.wall_mask & 2u)) ? bounce_moving<L, I>(p, 1, bb) : bb;
                 }
             }
         }
     }()),
     ...);
}

template <bool OUTF, class S, class L>
__device__ __forceinline__ void x_face_fixup(const Planes& pl, const KParams& p, int x, int y,
                                             int z, int s, unsigned lanes, bool cxm, bool cxp,
                                             int oym, int oyp, int ozm, int ozp, float* f,
                                             float* g) {
    if (!__any_sync(lanes, cxm || cxp)) return;  // interior warp
    const bool out = OUTF && !(p.wall_mask & 2u) && !(p.vel_mask & 2u);
    const int yz = y + p.ny * z;
    bool via[L::kQ];
#pragma unroll
    for (int i = 0; i < L::kQ; ++i) via[i] = false;
    x_face_f<OUTF, S, L>(pl, p, s, cxm, cxp, out, oym, oyp, ozm, ozp, yz, f, via,
                         std::make_integer_sequence<int, L::kQ>{});
    if (OUTF && cxp && out) outflow_anchor<L>(f, via);
    if (cxm) {  // x-low: wall / velocity face (an outflow is only allowed on x-high)
        const float bb = ldg_dev<S>(pl, p, 2, s);
        g[1] = p.heat_kind[0] == 2 ? -bb + p.heat_abb[0] : bb;
    }
    if (cxp) {
        const int kind = p.heat_kind[1];
        if (OUTF && kind == 3) {
            g[2] = outflow_blend(p, __ldg(pl.hin + 5 * p.nyz + chk(yz, p.nyz)), ldg_dev<S>(pl, p, 2, s));
        } else {
            const float bb = ldg_dev<S>(pl, p, 1, s);
            g[2] = kind == 2 ? -bb + p.heat_abb[1] : bb;
        }
    }
}

// Whether the y and z neighbours of a site need no face rule: they lie inside the ranges, or
// across a periodic face (faces are periodic in pairs), where the fast pull wraps the offset.
__device__ __forceinline__ bool yz_fast(const KParams& p, int y, int z) {
    const bool y_ok = (y > 0 && y < p.ny - 1) || (p.per_mask & 12u) == 12u;
    const bool z_ok = (z > 0 && z < p.nz - 1) || (p.per_mask & 48u) == 48u;
    return y_ok && z_ok;
}
// Whether no pull of a site crosses a non-periodic face.
__device__ __forceinline__ bool site_no_cross(const KParams& p, int x, int y, int z) {
    return yz_fast(p, y, z) && ((x > 0 && x < p.nx - 1) || (p.per_mask & 3u) == 3u);
}

// Source offsets of the six axis directions of a site (wrapped across periodic faces, 0 on a
// crossed face) and its crossing bits (x-low, x-high, y-low, y-high, z-low, z-high).
struct AxisOff {
    int xm, xp, ym, yp, zm, zp;
    unsigned cross;
};
__device__ __forceinline__ AxisOff axis_offsets(const KParams& p, int x, int y, int z) {
    const int nx = p.nx, nxy = p.nx * p.ny;
    AxisOff o;
    o.cross = 0u;
    o.xm = -1;
    o.xp = 1;
    o.ym = -nx;
    o.yp = nx;
    o.zm = -nxy;
    o.zp = nxy;
    if (x == 0) { if (p.per_mask & 1u) o.xm = nx - 1; else { o.xm = 0; o.cross |= 1u; } }
    if (x == nx - 1) { if (p.per_mask & 2u) o.xp = 1 - nx; else { o.xp = 0; o.cross |= 2u; } }
    if (y == 0) { if (p.per_mask & 4u) o.ym = nx * (p.ny - 1); else { o.ym = 0; o.cross |= 4u; } }
    if (y == p.ny - 1) { if (p.per_mask & 8u) o.yp = -nx * (p.ny - 1); else { o.yp = 0; o.cross |= 8u; } }
    if (z == 0) { if (p.per_mask & 16u) o.zm = nxy * (p.nz - 1); else { o.zm = 0; o.cross |= 16u; } }
    if (z == p.nz - 1) { if (p.per_mask & 32u) o.zp = -nxy * (p.nz - 1); else { o.zp = 0; o.cross |= 32u; } }
    return o;
}
template <int EX, int EY, int EZ>
__device__ __forceinline__ int src_off(const AxisOff& o) {
    return axis_off(EX, o.xm, o.xp) + axis_off(EY, o.ym, o.yp) + axis_off(EZ, o.zm, o.zp);
}
template <int EX, int EY, int EZ>
__device__ __forceinline__ unsigned src_cross(unsigned cr) {
    return axis_cross(EX, cr, 1u, 2u) | axis_cross(EY, cr, 4u, 8u) | axis_cross(EZ, cr, 16u, 32u);
}

// Pull of a site none of whose pulls crosses a non-periodic face: unconditional loads.
template <class S, class L = D3Q19>
__device__ __forceinline__ void gather_interior(const Planes& pl, const KParams& p, int x, int y,
                                                int z, int s, float* f, float* g) {
    const AxisOff o = axis_offsets(p, x, y, z);
#pragma unroll
    for (int i = 0; i < L::kQ; ++i)
        f[i] = ldp<S>(pl, p, i, s + axis_off(L::ex(i), o.xm, o.xp) + axis_off(L::ey(i), o.ym, o.yp) +
                                    axis_off(L::ez(i), o.zm, o.zp));
#pragma unroll
    for (int i = 0; i < kQT; ++i)
        g[i] = ldg_dev<S>(pl, p, i, s + axis_off(ex7(i), o.xm, o.xp) + axis_off(ey7(i), o.ym, o.yp) +
                                        axis_off(ez7(i), o.zm, o.zp));
}

// Load of plane I at idx, or of plane J (the opposite velocity, same weight) when `other`.
template <class S>
__device__ __forceinline__ float ldp_either(const Planes& pl, const KParams& p, int I, int J,
                                            bool other, int idx) {
    return S::ld(at_in_either<S>(pl, p, I, J, other, idx));
}
template <class S>
__device__ __forceinline__ float ldg_either(const Planes& pl, const KParams& p, int I, int J,
                                            bool other, int idx) {
    if constexpr (!S::kScaled) {
        return ldp_either<S>(pl, p, kQ + I, kQ + J, other, idx);
    } else {
        const float sc = I == 0 ? p.om0 : p.om1;
        return __fmul_rn(sc, __fmaf_rn(p.sigma, __ldg(pl.tin + chk(idx, p.ns)),
                                       S::ld(at_in_either<S>(pl, p, kQ + I, kQ + J, other, idx))));
    }
}

// Pull of any site of a lattice without node walls, with every load issued in one round: the
// source of each population is chosen per lane (the neighbour, the opposite plane of the site
// itself for a bounce-back, the inner source for the outflow), then the value rules of the
// crossed faces are applied to the loaded values.
template <bool OUTF, class S, class L, int... I>
__device__ __forceinline__ void sel_load_f(const Planes& pl, const KParams& p, int s,
                                           const AxisOff& o, float* f,
                                           std::integer_sequence<int, I...>) {
    (([&] {
         constexpr int ex = L::ex(I), ey = L::ey(I), ez = L::ez(I);
         const unsigned c = src_cross<ex, ey, ez>(o.cross);
         // the outflow rule reads plane I at the source with the x offset of the crossed
         // face (0), i.e. the inner neighbour's pull source; the other rules the opposite plane
         const bool bounce =
             c != 0u && !(OUTF && ex == -1 && !(c & (p.wall_mask | p.vel_mask)));
         f[I] = ldp_either<S>(pl, p, I, L::opp(I), bounce, bounce ? s : s + src_off<ex, ey, ez>(o));
     }()),
     ...);
}
template <bool OUTF, class S, class L, int... I>
__device__ __forceinline__ void sel_fix_f(const KParams& p, const AxisOff& o, const float* hf,
                                          float* f, bool* via, std::integer_sequence<int, I...>) {
    (([&] {
         constexpr int ex = L::ex(I), ey = L::ey(I), ez = L::ez(I);
         const unsigned c = src_cross<ex, ey, ez>(o.cross);
         via[I] = false;
         if (c != 0u && !(c & p.wall_mask)) {
             const unsigned vm = c & p.vel_mask;
             if (vm) {
                 f[I] = bounce_moving_on<L, I>(p, vm, f[I]);
             } else if constexpr (OUTF && ex == -1) {
                 f[I] = outflow_blend(p, hf[L::slot(I)], f[I]);
                 via[I] = true;
             }
         }
     }()),
     ...);
}
template <int... I>
__device__ __forceinline__ void sel_fix_g(const KParams& p, const AxisOff& o, bool gout,
                                          const float* hf, float* g,
                                          std::integer_sequence<int, I...>) {
    (([&] {
         const unsigned c = src_cross<ex7(I), ey7(I), ez7(I)>(o.cross);
         if (c == 0u) return;
         constexpr int face = face7(I);
         if (I == 2 && gout) g[I] = outflow_blend(p, hf[5], g[I]);
         else if (p.heat_kind[face] == 2) g[I] = -g[I] + p.heat_abb[face];  // anti-bounce-back
     }()),
     ...);
}

template <bool OUTF, class S, class L>
__device__ __forceinline__ void gather_sel(const Planes& pl, const KParams& p, int x, int y, int z,
                                           int s, float* f, float* g) {
    const AxisOff o = axis_offsets(p, x, y, z);
    sel_load_f<OUTF, S, L>(pl, p, s, o, f, std::make_integer_sequence<int, L::kQ>{});
    // D3Q7: one face at most per velocity; the outflow rule (x-high, kind 3) reads plane 2 at
    // the site itself, the other rules the opposite plane of the site
    const bool gout = OUTF && (o.cross & 2u) && p.heat_kind[1] == 3;
#pragma unroll
    for (int i = 0; i < kQT; ++i) {
        const unsigned c = axis_cross(ex7(i), o.cross, 1u, 2u) | axis_cross(ey7(i), o.cross, 4u, 8u) |
                           axis_cross(ez7(i), o.cross, 16u, 32u);
        const bool bounce = c != 0u && !(i == 2 && gout);
        g[i] = ldg_either<S>(pl, p, i, opp7(i), bounce,
                             c != 0u ? s : s + axis_off(ex7(i), o.xm, o.xp) +
                                               axis_off(ey7(i), o.ym, o.yp) +
                                               axis_off(ez7(i), o.zm, o.zp));
    }
    float hf[kOutSlots];  // outflow history of the lanes on the x-high face, same round
    if constexpr (OUTF) {
        const bool xo = (o.cross & 2u) != 0u;
        const int yz = y + p.ny * z;
#pragma unroll
        for (int k = 0; k < kOutSlots; ++k) hf[k] = xo ? __ldg(pl.hin + k * p.nyz + chk(yz, p.nyz)) : 0.0f;
    }
    if (o.cross == 0u) return;  // no face rule at this site
    bool via[L::kQ];
    sel_fix_f<OUTF, S, L>(p, o, hf, f, via, std::make_integer_sequence<int, L::kQ>{});
    if (OUTF && (o.cross & 2u)) outflow_anchor<L>(f, via);
    sel_fix_g(p, o, gout, hf, g, std::make_integer_sequence<int, kQT>{});
}

// ---- collision -------------------------------------------------------------------------------
// Eqs. B8-B9: temperature and liquid fraction from the effective enthalpy.
__device__ __forceinline__ void enthalpy_state(const KParams& p, float En, float& T, float& fl) {
    if (En <= p.ent_Es) {
        T = __fmul_rn(En, p.ent_is);
        fl = 0.0f;
    } else if (En >= p.ent_El) {
        T = __fmaf_rn(__fsub_rn(En, p.ent_El), p.ent_il, p.ent_Tl);
        fl = 1.0f;
    } else {
        fl = __fmul_rn(__fsub_rn(En, p.ent_Es), p.ent_idE);
        T = __fmaf_rn(fl, __fsub_rn(p.ent_Tl, p.ent_Ts), p.ent_Ts);
    }
}

template <class V>
struct MacroT {
    V rho, ux, uy, uz, T, dT;  // dT = T - T0
};
struct Macro {
    float rho, ux, uy, uz, T, dT;  // dT = T - T0
};

// D3Q7: n = N g (Eq. 36), n_eq = T (sigma, u, varpi sigma, 0, 0) (Eq. 37), Eq. 34, Eq. 43;
// enthalpy model (one site at a time): n_eq = (En_e, c_pl T u, varpi c_ref T, 0, 0) (Eq. B6)
// on full values, zeta_alpha from Eq. B11 with alpha_e = f_l alpha_l + (1 - f_l) alpha_s.
// n0 = sum g (the deviation sigma (T - T0), or En_e), u the flow's velocity; g is updated in
// place.
template <class V, bool ENTH>
__device__ __forceinline__ void collide_g_t(const KParams& p, const MediumT<V>& md, V* g, V n0, V T,
                                            float fl, V ux, V uy, V uz) {
    const V g12 = g[1] + g[2], g34 = g[3] + g[4], g56 = g[5] + g[6];
    const V n4 = (g12 + g34) + g56;  // minus varpi sigma T0 (standard model)
    V tu = T, n4eq = K<V>(p.varpi) * n0, za = md.zeta_alpha;
    if constexpr (ENTH) {
        tu = K<V>(p.c_pl) * T;
        n4eq = K<V>(__fmul_rn(p.varpi, p.c_ref)) * T;
        za = K<V>(__fdividef(1.0f, __fmaf_rn(__fmaf_rn(fl, p.alpha_l,
                                                       __fmul_rn(__fsub_rn(1.0f, fl), p.alpha_s)),
                                             p.inv_csT2, 0.5f)));
    }
    const V dn1 = za * fma(tu, ux, -(g[1] - g[2]));
    const V dn2 = za * fma(tu, uy, -(g[3] - g[4]));
    const V dn3 = za * fma(tu, uz, -(g[5] - g[6]));
    const V c4 = K<V>(p.ze6) * (n4eq - n4);   // dn4 / 6
    const V c5 = K<V>(-p.zn6) * (g12 - g34);  // dn5 / 6
    const V c6 = K<V>(-p.zn6) * (g12 - g56);  // dn6 / 6
    g[0] = fma(K<V>(-6.0f), c4, g[0]);
    const V c46 = c4 + c6;
    const V gx = c46 + c5, gy = fma(K<V>(-2.0f), c5, c46), gz = fma(K<V>(-2.0f), c6, c4 + c5);
    const V h1 = K<V>(0.5f) * dn1, h2 = K<V>(0.5f) * dn2, h3 = K<V>(0.5f) * dn3;
    g[1] = g[1] + (gx + h1);
    g[2] = g[2] + (gx - h1);
    g[3] = g[3] + (gy + h2);
    g[4] = g[4] + (gy - h2);
    g[5] = g[5] + (gz + h3);
    g[6] = g[6] + (gz - h3);
}
template <bool ENTH>
__device__ __forceinline__ void collide_g(const KParams& p, const Medium& md, float* g, float n0,
                                          float T, float fl, float ux, float uy, float uz) {
    collide_g_t<L1, ENTH>(p, md, reinterpret_cast<L1*>(g), L1{n0}, L1{T}, fl, L1{ux}, L1{uy},
                          L1{uz});
}

// Eqs. 39, 5, 25, 27-28, 4, then (FULL) Eq. 9 with Eqs. 21-23 in moment space and Eq. 34 with
// Eqs. 37-38, back-transformed in place, on one site (L1) or a pair (L2).  f, g are
// deviations on entry and exit.  The per-moment factors s_k / |M_k|^2 and (1 - s_k/2) /
// |M_k|^2 come precomputed in KParams.  PU (one site): the velocity is prescribed (pu, a node
// wall) instead of solved from Eqs. 27-28, and the conserved momentum becomes
// rho0 pu + rho0 F / 2 after the collision.  ENTH (one site): the enthalpy model.
// GOut: called as gout(g, dT) with the post-collision D3Q7 populations as soon as they are
// final (the thermal collision needs only T and u), so that a caller can store them before
// the D3Q19 relaxation runs and its registers are free; NoGStore leaves them in g.
struct NoGStore {
    template <class V>
    __device__ __forceinline__ void operator()(const V*, V) const {}
};
template <class V, bool FULL, bool ENTH = false, bool PU = false, class GOut = NoGStore>
__device__ __forceinline__ MacroT<V> collide_t(const KParams& p, const MediumT<V>& md, V* f, V* g,
                                               float pux = 0.0f, float puy = 0.0f,
                                               float puz = 0.0f, GOut gout = GOut{}) {
    static_assert(std::is_same<V, L1>::value || !(ENTH || PU), "paired sites: standard model");
    // temperature (Eq. 39, or Eqs. B7-B9 with the enthalpy model) and body force (Eq. 5)
    const V n0 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);  // sigma (T - T0)
    V T, dT;                                                                 // or En_e
    float fl = 1.0f;
    if constexpr (ENTH) {
        float t;
        enthalpy_state(p, n0.v, t, fl);
        T = L1{t};
        dT = L1{__fsub_rn(t, p.T0)};
    } else {
        dT = n0 * K<V>(p.inv_sigma);
        T = K<V>(p.T0) + dT;
    }
    const V Gx = fma(K<V>(p.buoy[0]), dT, K<V>(p.accel[0]));
    const V Gy = fma(K<V>(p.buoy[1]), dT, K<V>(p.accel[1]));
    const V Gz = fma(K<V>(p.buoy[2]), dT, K<V>(p.accel[2]));

    // symmetric / antisymmetric sums over opposite pairs
    const V s1 = f[1] + f[2], d1 = f[1] - f[2];
    const V s2 = f[3] + f[4], d2 = f[3] - f[4];
    const V s3 = f[5] + f[6], d3 = f[5] - f[6];
    const V s4 = f[7] + f[10], d4 = f[7] - f[10];   // ( 1, 1, 0)
    const V s5 = f[8] + f[9], d5 = f[8] - f[9];     // (-1, 1, 0)
    const V s6 = f[11] + f[14], d6 = f[11] - f[14]; // ( 1, 0, 1)
    const V s7 = f[12] + f[13], d7 = f[12] - f[13]; // (-1, 0, 1)
    const V s8 = f[15] + f[18], d8 = f[15] - f[18]; // ( 0, 1, 1)
    const V s9 = f[16] + f[17], d9 = f[16] - f[17]; // ( 0,-1, 1)
    const V A = (s1 + s2) + s3;
    const V Dxy = s4 + s5, Dxz = s6 + s7, Dyz = s8 + s9;
    const V D = (Dxy + Dxz) + Dyz;
    const V rho = (f[0] + A) + D;  // rho - rho0 (Eq. 25)
    const V d45 = d4 - d5, d67 = d6 - d7, d89 = d8 - d9;
    const V e45 = d4 + d5, e67 = d6 + d7, e89 = d8 + d9;
    const V jx = (d1 + d45) + d67;
    const V jy = (d2 + e45) + d89;
    const V jz = (d3 + e67) + e89;

    // velocity (Eqs. 27-28) and total force (Eq. 4)
    const V hphi = K<V>(0.5f) * md.phi;
    const V vx = fma(jx, K<V>(p.inv_rho0), hphi * Gx);
    const V vy = fma(jy, K<V>(p.inv_rho0), hphi * Gy);
    const V vz = fma(jz, K<V>(p.inv_rho0), hphi * Gz);
    const V vmag = lanes(fma(vz, vz, fma(vy, vy, vx * vx)), sqrt_nonneg);
    const V root = lanes(fma(md.l1, vmag, md.l0 * md.l0), sqrt_nonneg);
    const V inv_den = lanes(md.l0 + root, [](float d) { return __fdividef(1.0f, d); });
    V ux = vx * inv_den, uy = vy * inv_den, uz = vz * inv_den;
    if constexpr (PU) {
        ux = L1{pux};
        uy = L1{puy};
        uz = L1{puz};
    }
    // enthalpy model: the flow is collided only where f_l >= 0.5; elsewhere u = 0
    bool rest = false;
    if constexpr (ENTH) {
        rest = p.flow_off || fl < 0.5f;
        if (rest) ux = uy = uz = L1{0.0f};
    }

    MacroT<V> mac;
    mac.rho = K<V>(p.rho0) + rho * K<V>(p.inv_fu);
    mac.ux = ux;
    mac.uy = uy;
    mac.uz = uz;
    mac.T = T;
    mac.dT = dT;
    if (!FULL) return mac;

    collide_g_t<V, ENTH>(p, md, g, n0, T, fl, ux, uy, uz);
    gout(static_cast<const V*>(g), dT);

    if (rest) {  // f_eq(rho, 0) in deviation form: w_i (rho - rho0)
#pragma unroll
        for (int i = 0; i < kQ; ++i) f[i] = K<V>(w19(i)) * rho;
    } else {
    // |u| = |v| / (l0 + sqrt(l0^2 + l1 |v|))
    V umag;
    if constexpr (PU) umag = lanes(fma(uz, uz, fma(uy, uy, ux * ux)), sqrt_nonneg);
    else umag = vmag * inv_den;
    const V drag = fma(md.c_forch, umag, md.c_darcy);
    const V Fx = fma(md.phi, Gx, -(drag * ux));
    const V Fy = fma(md.phi, Gy, -(drag * uy));
    const V Fz = fma(md.phi, Gz, -(drag * uz));

    // moments of Eq. 20 (rows of Eq. A2) that relax
    const V m_e = fma(K<V>(-30.0f), f[0], fma(K<V>(-11.0f), A, K<V>(8.0f) * D));
    const V m_eps = fma(K<V>(12.0f), f[0], fma(K<V>(-4.0f), A, D));
    const V qx = fma(K<V>(-5.0f), d1, jx), qy = fma(K<V>(-5.0f), d2, jy),
            qz = fma(K<V>(-5.0f), d3, jz);
    const V s23 = s2 + s3;
    const V Dw = fma(K<V>(-2.0f), Dyz, Dxy + Dxz);  // Dxy + Dxz - 2 Dyz
    const V m_pxx = fma(K<V>(2.0f), s1, Dw - s23);
    const V m_pixx = fma(K<V>(-4.0f), s1, fma(K<V>(2.0f), s23, Dw));
    const V Dv = Dxy - Dxz;
    const V m_pww = (s2 - s3) + Dv;
    const V m_piww = fma(K<V>(2.0f), s3 - s2, Dv);
    const V m_pxy = s4 - s5, m_pyz = s8 - s9, m_pzx = s6 - s7;
    const V m_mx = d45 - d67;
    const V m_my = d89 - e45;
    const V m_mz = e67 - e89;

    // equilibria (Eq. 21, beta1 = 3, beta2 = -11/2, beta3 = -1/2) and forcing (Eq. 23), with
    // the velocity scaled by rho0 / phi once: w = rho0 u / phi
    const V r0p = K<V>(p.frho0) * md.inv_phi;
    const V wx = r0p * ux, wy = r0p * uy, wz = r0p * uz;
    const V pxx = wx * ux, pyy = wy * uy, pzz = wz * uz;  // rho0 u_a^2 / phi
    const V fxx = wx * Fx, fyy = wy * Fy, fzz = wz * Fz;  // rho0 u_a F_a / phi
    const V usq = (pxx + pyy) + pzz;
    const V uF = (fxx + fyy) + fzz;
    const V pyz = pyy + pzz, fyz = fyy + fzz;
    const V eq_pxx = fma(K<V>(2.0f), pxx, -pyz);
    const V eq_pww = pyy - pzz;
    const V S_pxx = K<V>(2.0f) * fma(K<V>(2.0f), fxx, -fyz);
    const V S_pww = K<V>(2.0f) * (fyy - fzz);

    // dm_k / |M_k|^2 = -s_k (m_k - m_k^eq) / |M_k|^2 + (1 - s_k/2) S_k / |M_k|^2; the conserved
    // momentum gains rho0 F whatever s_j is (Eqs. 9, 14, 26)
    const V de = fma(K<V>(p.ae), fma(K<V>(-11.0f), rho, fma(K<V>(19.0f), usq, -m_e)),
                     K<V>(__fmul_rn(38.0f, p.be)) * uF);
    const V deps = fma(K<V>(p.aeps), fma(K<V>(3.0f), rho, fma(K<V>(-5.5f), usq, -m_eps)),
                       K<V>(__fmul_rn(-11.0f, p.beps)) * uF);
    V djx = K<V>(p.rho0_10) * Fx, djy = K<V>(p.rho0_10) * Fy, djz = K<V>(p.rho0_10) * Fz;
    if constexpr (PU) {
        djx = K<V>(0.1f) * fma(K<V>(p.frho0), fma(K<V>(0.5f), Fx, ux), -jx);
        djy = K<V>(0.1f) * fma(K<V>(p.frho0), fma(K<V>(0.5f), Fy, uy), -jy);
        djz = K<V>(0.1f) * fma(K<V>(p.frho0), fma(K<V>(0.5f), Fz, uz), -jz);
    }
    const V dqx = fma(K<V>(-p.aq), qx, -fma(K<V>(p.aqc), ux, K<V>(p.bqc) * Fx));
    const V dqy = fma(K<V>(-p.aq), qy, -fma(K<V>(p.aqc), uy, K<V>(p.bqc) * Fy));
    const V dqz = fma(K<V>(-p.aq), qz, -fma(K<V>(p.aqc), uz, K<V>(p.bqc) * Fz));
    const V dpxx = fma(K<V>(p.anu36), eq_pxx - m_pxx, K<V>(p.bnu36) * S_pxx);
    const V dpixx = fma(K<V>(-p.api72), fma(K<V>(0.5f), eq_pxx, m_pixx), K<V>(-p.hbpi72) * S_pxx);
    const V dpww = fma(K<V>(p.anu12), eq_pww - m_pww, K<V>(p.bnu12) * S_pww);
    const V dpiww = fma(K<V>(-p.api24), fma(K<V>(0.5f), eq_pww, m_piww), K<V>(-p.hbpi24) * S_pww);
    const V dpxy = fma(K<V>(p.anu4), fma(wx, uy, -m_pxy), K<V>(p.bnu4) * fma(wx, Fy, wy * Fx));
    const V dpyz = fma(K<V>(p.anu4), fma(wy, uz, -m_pyz), K<V>(p.bnu4) * fma(wy, Fz, wz * Fy));
    const V dpzx = fma(K<V>(p.anu4), fma(wz, ux, -m_pzx), K<V>(p.bnu4) * fma(wz, Fx, wx * Fz));
    const V dmx = K<V>(-p.am8) * m_mx;
    const V dmy = K<V>(-p.am8) * m_my;
    const V dmz = K<V>(-p.am8) * m_mz;

    // f* = f + M^T diag(1/|M_k|^2) dm
    f[0] = f[0] + fma(K<V>(-30.0f), de, K<V>(12.0f) * deps);
    const V Eax = fma(K<V>(-11.0f), de, K<V>(-4.0f) * deps);
    const V Ex = fma(K<V>(2.0f), dpxx, fma(K<V>(-4.0f), dpixx, Eax));
    const V Eyz2 = fma(K<V>(2.0f), dpixx, Eax - dpxx);
    const V Pw = fma(K<V>(-2.0f), dpiww, dpww);
    const V Ey = Eyz2 + Pw;
    const V Ez = Eyz2 - Pw;
    const V Ox = fma(K<V>(-4.0f), dqx, djx), Oy = fma(K<V>(-4.0f), dqy, djy),
            Oz = fma(K<V>(-4.0f), dqz, djz);
    f[1] = f[1] + (Ex + Ox);
    f[2] = f[2] + (Ex - Ox);
    f[3] = f[3] + (Ey + Oy);
    f[4] = f[4] + (Ey - Oy);
    f[5] = f[5] + (Ez + Oz);
    f[6] = f[6] + (Ez - Oz);
    const V Cd = fma(K<V>(8.0f), de, deps);
    const V pp = dpxx + dpixx;
    const V Cp = Cd + pp;
    const V Pww = dpww + dpiww;
    const V Exy = Cp + Pww;
    const V Exz = Cp - Pww;
    const V Eyz = fma(K<V>(-2.0f), pp, Cd);
    const V Jx = djx + dqx, Jy = djy + dqy, Jz = djz + dqz;
    const V mxy = dmx - dmy, mxz = dmz - dmx, myz = dmy - dmz;
    const V O7 = (Jx + Jy) + mxy;
    const V O8 = (Jy - Jx) - (dmx + dmy);
    const V O11 = (Jx + Jz) + mxz;
    const V O12 = (Jz - Jx) + (dmx + dmz);
    const V O15 = (Jy + Jz) + myz;
    const V O16 = (Jz - Jy) - (dmy + dmz);
    const V Ea = Exy + dpxy, Eb = Exy - dpxy;
    const V Ec = Exz + dpzx, Ed = Exz - dpzx;
    const V Ee = Eyz + dpyz, Ef = Eyz - dpyz;
    f[7] = f[7] + (Ea + O7);
    f[10] = f[10] + (Ea - O7);
    f[8] = f[8] + (Eb + O8);
    f[9] = f[9] + (Eb - O8);
    f[11] = f[11] + (Ec + O11);
    f[14] = f[14] + (Ec - O11);
    f[12] = f[12] + (Ed + O12);
    f[13] = f[13] + (Ed - O12);
    f[15] = f[15] + (Ee + O15);
    f[18] = f[18] + (Ee - O15);
    f[16] = f[16] + (Ef + O16);
    f[17] = f[17] + (Ef - O16);

    }  // flow collision

    return mac;
}
template <bool FULL, bool ENTH = false, bool PU = false, class GOut = NoGStore>
__device__ __forceinline__ Macro collide(const KParams& p, const Medium& md, float* f, float* g,
                                         float pux = 0.0f, float puy = 0.0f, float puz = 0.0f,
                                         GOut gout = GOut{}) {
    const MacroT<L1> m = collide_t<L1, FULL, ENTH, PU>(p, md, reinterpret_cast<L1*>(f),
                                                       reinterpret_cast<L1*>(g), pux, puy, puz,
                                                       gout);
    return {m.rho.v, m.ux.v, m.uy.v, m.uz.v, m.T.v, m.dT.v};
}

// D3Q15 (Sec. 3.1.1): the same steps with the moments of Eq. 13 (rows of Eq. A1), the
// equilibria of Eq. 15 (beta1 = 1, beta2 = -5), the forcing of Eq. 17 and Lambda of Eq. 16,
// back-transformed through M^T diag(1/|M_k|^2) (the rows of Eq. A1 are orthogonal, with
// |M_k|^2 = 15, 18, 360, 10, 40, 12, 4, 8).  f, g are deviations on entry and exit.
template <bool FULL, bool PU = false>
__device__ __forceinline__ Macro collide15(const KParams& p, const Medium& md, float* f, float* g,
                                           float pux = 0.0f, float puy = 0.0f, float puz = 0.0f) {
    const float n0 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);  // sigma (T - T0)
    const float dT = __fmul_rn(n0, p.inv_sigma);  // rounded product, as in collide
    const float T = p.T0 + dT;
    const float Gx = p.buoy[0] * dT + p.accel[0];
    const float Gy = p.buoy[1] * dT + p.accel[1];
    const float Gz = p.buoy[2] * dT + p.accel[2];

    // sums / differences over opposite pairs; the four corner pairs along (+-1, +-1, 1)
    const float s1 = f[1] + f[2], d1 = f[1] - f[2];
    const float s2 = f[3] + f[4], d2 = f[3] - f[4];
    const float s3 = f[5] + f[6], d3 = f[5] - f[6];
    const float sa = f[7] + f[14], da = f[7] - f[14];    // ( 1, 1, 1)
    const float sb = f[8] + f[13], db = f[8] - f[13];    // (-1, 1, 1)
    const float sc = f[9] + f[12], dc = f[9] - f[12];    // ( 1,-1, 1)
    const float sd = f[10] + f[11], dd = f[10] - f[11];  // (-1,-1, 1)
    const float A = s1 + s2 + s3;
    const float Cs = (sa + sb) + (sc + sd);
    const float rho = f[0] + A + Cs;  // rho - rho0 (Eq. 25)
    const float jx = d1 + (da - db) + (dc - dd);
    const float jy = d2 + (da + db) - (dc + dd);
    const float jz = d3 + (da + db) + (dc + dd);

    // velocity (Eqs. 27-28) and total force (Eq. 4)
    const float hphi = 0.5f * md.phi.v;
    const float vx = jx * p.inv_rho0 + hphi * Gx;
    const float vy = jy * p.inv_rho0 + hphi * Gy;
    const float vz = jz * p.inv_rho0 + hphi * Gz;
    const float vmag = sqrt_nonneg(vx * vx + vy * vy + vz * vz);
    const float inv_den = __fdividef(1.0f, md.l0.v + sqrt_nonneg(md.l0.v * md.l0.v + md.l1.v * vmag));
    const float ux = PU ? pux : vx * inv_den, uy = PU ? puy : vy * inv_den;
    const float uz = PU ? puz : vz * inv_den;

    Macro mac;
    mac.rho = p.rho0 + rho;
    mac.ux = ux;
    mac.uy = uy;
    mac.uz = uz;
    mac.T = T;
    mac.dT = dT;
    if (!FULL) return mac;

    const float umag = PU ? sqrt_nonneg(ux * ux + uy * uy + uz * uz) : vmag * inv_den;
    const float drag = md.c_darcy.v + md.c_forch.v * umag;
    const float Fx = md.phi.v * Gx - drag * ux;
    const float Fy = md.phi.v * Gy - drag * uy;
    const float Fz = md.phi.v * Gz - drag * uz;

    // moments of Eq. 13 (rows of Eq. A1) that relax
    const float m_e = -2.0f * f[0] - A + Cs;
    const float m_eps = 16.0f * f[0] - 4.0f * A + Cs;
    const float qx = jx - 5.0f * d1, qy = jy - 5.0f * d2, qz = jz - 5.0f * d3;
    const float m_pxx = 2.0f * s1 - s2 - s3;
    const float m_pww = s2 - s3;
    const float m_pxy = (sa + sd) - (sb + sc);
    const float m_pyz = (sa + sb) - (sc + sd);
    const float m_pzx = (sa + sc) - (sb + sd);
    const float m_xyz = (da + dd) - (db + dc);

    // equilibria (Eq. 15) and forcing (Eq. 17) with w = rho0 u / phi
    const float r0p = p.rho0 * md.inv_phi.v;
    const float wx = r0p * ux, wy = r0p * uy, wz = r0p * uz;
    const float pxx = wx * ux, pyy = wy * uy, pzz = wz * uz;
    const float fxx = wx * Fx, fyy = wy * Fy, fzz = wz * Fz;
    const float usq = pxx + pyy + pzz;
    const float uF = fxx + fyy + fzz;
    const float eq_pxx = 2.0f * pxx - pyy - pzz;
    const float eq_pww = pyy - pzz;
    const float S_pxx = 2.0f * (2.0f * fxx - fyy - fzz);
    const float S_pww = 2.0f * (fyy - fzz);

    // dm_k / |M_k|^2 (Eq. 9); the conserved momentum gains rho0 F whatever s_j is
    const float de = p.ae15 * (usq - rho - m_e) + p.be15 * 2.0f * uF;
    const float deps = p.aeps15 * (rho - 5.0f * usq - m_eps) - p.beps15 * 10.0f * uF;
    float djx = p.rho0_10 * Fx, djy = p.rho0_10 * Fy, djz = p.rho0_10 * Fz;
    if constexpr (PU) {
        djx = 0.1f * (p.rho0 * (ux + 0.5f * Fx) - jx);
        djy = 0.1f * (p.rho0 * (uy + 0.5f * Fy) - jy);
        djz = 0.1f * (p.rho0 * (uz + 0.5f * Fz) - jz);
    }
    const float dqx = -p.aq * qx - (p.aqc15 * ux + p.bqc15 * Fx);
    const float dqy = -p.aq * qy - (p.aqc15 * uy + p.bqc15 * Fy);
    const float dqz = -p.aq * qz - (p.aqc15 * uz + p.bqc15 * Fz);
    const float dpxx = p.anu12 * (eq_pxx - m_pxx) + p.bnu12 * S_pxx;
    const float dpww = p.anu4 * (eq_pww - m_pww) + p.bnu4 * S_pww;
    const float dpxy = p.anu8 * (wx * uy - m_pxy) + p.bnu8 * (wx * Fy + wy * Fx);
    const float dpyz = p.anu8 * (wy * uz - m_pyz) + p.bnu8 * (wy * Fz + wz * Fy);
    const float dpzx = p.anu8 * (wz * ux - m_pzx) + p.bnu8 * (wz * Fx + wx * Fz);
    const float dm = -p.am8 * m_xyz;

    // f* = f + M^T diag(1/|M_k|^2) dm (columns of Eq. A1)
    f[0] += -2.0f * de + 16.0f * deps;
    const float Ea = -de - 4.0f * deps;
    const float Ex = Ea + 2.0f * dpxx;
    const float Ey = Ea - dpxx + dpww;
    const float Ez = Ea - dpxx - dpww;
    const float Ox = djx - 4.0f * dqx, Oy = djy - 4.0f * dqy, Oz = djz - 4.0f * dqz;
    f[1] += Ex + Ox;
    f[2] += Ex - Ox;
    f[3] += Ey + Oy;
    f[4] += Ey - Oy;
    f[5] += Ez + Oz;
    f[6] += Ez - Oz;
    const float Cc = de + deps;
    const float Jx = djx + dqx, Jy = djy + dqy, Jz = djz + dqz;
    const float E7 = Cc + dpxy + dpyz + dpzx, O7 = Jx + Jy + Jz + dm;     // ( 1, 1, 1)
    const float E8 = Cc - dpxy + dpyz - dpzx, O8 = -Jx + Jy + Jz - dm;    // (-1, 1, 1)
    const float E9 = Cc - dpxy - dpyz + dpzx, O9 = Jx - Jy + Jz - dm;     // ( 1,-1, 1)
    const float E10 = Cc + dpxy - dpyz - dpzx, O10 = -Jx - Jy + Jz + dm;  // (-1,-1, 1)
    f[7] += E7 + O7;
    f[14] += E7 - O7;
    f[8] += E8 + O8;
    f[13] += E8 - O8;
    f[9] += E9 + O9;
    f[12] += E9 - O9;
    f[10] += E10 + O10;
    f[11] += E10 - O10;

    collide_g<false>(p, md, g, n0, T, 1.0f, ux, uy, uz);
    return mac;
}

// The collision of the flow lattice L (PU: with the velocity prescribed as pu).
template <bool FULL, bool ENTH, class L, bool PU = false, class GOut = NoGStore>
__device__ __forceinline__ Macro collide_on(const KParams& p, const Medium& md, float* f, float* g,
                                            float pux = 0.0f, float puy = 0.0f, float puz = 0.0f,
                                            GOut gout = GOut{}) {
    if constexpr (L::kQ == 15) {
        const Macro m = collide15<FULL, PU>(p, md, f, g, pux, puy, puz);
        if (FULL) gout(reinterpret_cast<const L1*>(g), L1{m.dT});
        return m;
    } else {
        return collide<FULL, ENTH, PU>(p, md, f, g, pux, puy, puz, gout);
    }
}

// ---- node walls (non-equilibrium extrapolation) -------------------------------------------------
// Node-wall faces a site lies on (bit f for face f).
__device__ __forceinline__ unsigned nee_bits(const KParams& p, int x, int y, int z) {
    unsigned b = 0u;
    if (x == 0) b |= p.nee_mask & 1u;
    if (x == p.nx - 1) b |= p.nee_mask & 2u;
    if (y == 0) b |= p.nee_mask & 4u;
    if (y == p.ny - 1) b |= p.nee_mask & 8u;
    if (z == 0) b |= p.nee_mask & 16u;
    if (z == p.nz - 1) b |= p.nee_mask & 32u;
    return b;
}

// A node-wall site (faces `nb`): the wall equilibrium plus the streamed non-equilibrium part
// of the fluid site beside it (Guo's rule), collided at the wall's own state with the velocity
// prescribed as u_w; rho_b = rho_f, or rho0 on a wall that withdraws fluid.  On exit f, g hold
// the post-collision populations of the wall site; the returned macros are (rho_b, u_w, T_b).
template <bool HET, bool FULL, class S, class L>
__device__ __forceinline__ Macro nee_site(const Planes& pl, const KParams& p, int x, int y, int z,
                                          int s, unsigned nb, float* f, float* g) {
    int c[3] = {x, y, z};
    int wall = -1, hot = -1;
#pragma unroll
    for (int fc = 0; fc < 6; ++fc)
        if (nb & (1u << fc)) {
            c[fc >> 1] += (fc & 1) ? -1 : 1;
            if (wall < 0) wall = fc;
            if (hot < 0 && p.heat_kind[fc] == 4) hot = fc;
        }
    const Nbr n = neighbourhood(p, c[0], c[1], c[2]);
    gather_general<false, S, L>(pl, p, n, f, g);
    const Medium mf = medium_at<HET>(p, n.s);
    const Macro m = collide_on<false, false, L>(p, mf, f, g);  // macros of x_f; f, g unchanged
    const float uwx = p.face_u[wall][0], uwy = p.face_u[wall][1], uwz = p.face_u[wall][2];
    const float dTb = hot >= 0 ? p.face_dT[hot] : m.dT;
    const float outw = (wall & 1) ? p.face_u[wall][wall >> 1] : -p.face_u[wall][wall >> 1];
    const float drf = m.rho - p.rho0;
    const float drb = outw > 0.0f ? 0.0f : drf;
    const Medium mb = medium_at<HET>(p, s);
    // f += f_eq(rho_b, u_w) - f_eq(rho_f, u_f) (Eqs. 18, 24), deviations
    const float iub = (uwx * uwx + uwy * uwy + uwz * uwz) * mb.inv_phi.v;
    const float iuf = (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz) * mf.inv_phi.v;
#pragma unroll
    for (int i = 0; i < L::kQ; ++i) {
        const float ebu = (float)L::ex(i) * uwx + (float)L::ey(i) * uwy + (float)L::ez(i) * uwz;
        const float efu = (float)L::ex(i) * m.ux + (float)L::ey(i) * m.uy + (float)L::ez(i) * m.uz;
        f[i] += L::w(i) * ((drb - drf) +
                           p.rho0 * (3.0f * (ebu - efu) + 4.5f * (ebu * ebu * mb.inv_phi.v - efu * efu * mf.inv_phi.v) -
                                     1.5f * (iub - iuf)));
    }
    // g += g_eq(T_b, u_w) - g_eq(T_f, u_f) (Eq. 42), deviations from omega_i sigma T0
    const float Tb = p.T0 + dTb;
    g[0] += p.om0 * p.sigma * (dTb - m.dT);
#pragma unroll
    for (int i = 1; i < kQT; ++i) {
        const float ebu = (float)ex7(i) * uwx + (float)ey7(i) * uwy + (float)ez7(i) * uwz;
        const float efu = (float)ex7(i) * m.ux + (float)ey7(i) * m.uy + (float)ez7(i) * m.uz;
        g[i] += p.om1 * p.sigma * (dTb - m.dT) + 0.5f * (ebu * Tb - efu * m.T);
    }
    Macro mac;
    mac.rho = p.rho0 + drb;
    mac.ux = uwx;
    mac.uy = uwy;
    mac.uz = uwz;
    mac.T = Tb;
    mac.dT = dTb;
    if constexpr (FULL) collide_on<true, false, L, true>(p, mb, f, g, uwx, uwy, uwz);
    return mac;
}

// ---- kernels ---------------------------------------------------------------------------------
// Pull of a site whose y and z neighbours need no rule (yz_fast) but which may lie on a
// non-periodic x face: the populations with e_x = 0 are plain loads; those with e_x = +1
// (-1) read the opposite plane of the site itself on a lane at the x-low (x-high) face, or,
// for the outflow, plane I at the inner source.  One round of loads, then the rules of the
// two x faces, whose parameters are compile-time entries of the parameter block.
template <bool OUTF, class S, class L, int... I>
__device__ __forceinline__ void xsel_load_f(const Planes& pl, const KParams& p, int s,
                                            const AxisOff& o, bool cxm, bool cxp, bool xout,
                                            float* f, std::integer_sequence<int, I...>) {
    (([&] {
         constexpr int ex = L::ex(I), ey = L::ey(I), ez = L::ez(I);
         const int src = s + src_off<ex, ey, ez>(o);
         if constexpr (ex == 0) {
             f[I] = ldp<S>(pl, p, I, src);
         } else {
             const bool bounce = ex == 1 ? cxm : (cxp && !xout);
             f[I] = ldp_either<S>(pl, p, I, L::opp(I), bounce, bounce ? s : src);
         }
     }()),
     ...);
}
template <bool OUTF, class S, class L, int... I>
__device__ __forceinline__ void xsel_fix_f(const KParams& p, bool cxm, bool cxp, bool xout,
                                           const float* hf, float* f, bool* via,
                                           std::integer_sequence<int, I...>) {
    const bool vlo = (p.vel_mask & 1u) && !(p.wall_mask & 1u);
    const bool vhi = (p.vel_mask & 2u) && !(p.wall_mask & 2u);
    (([&] {
         constexpr int ex = L::ex(I);
         via[I] = false;
         if constexpr (ex == 1) {
             if (cxm && vlo) f[I] = bounce_moving<L, I>(p, 0, f[I]);
         } else if constexpr (ex == -1) {
             if (cxp) {
                 if (xout) {
                     if constexpr (OUTF) {
                         f[I] = outflow_blend(p, hf[L::slot(I)], f[I]);
                         via[I] = true;
                     }
                 } else if (vhi) {
                     f[I] = bounce_moving<L, I>(p, 1, f[I]);
                 }
             }
         }
     }()),
     ...);
}
template <bool OUTF, class S, class L>
__device__ __forceinline__ void gather_xsel(const Planes& pl, const KParams& p, int x, int y,
                                            int z, int s, float* f, float* g) {
    const AxisOff o = axis_offsets(p, x, y, z);
    const bool cxm = (o.cross & 1u) != 0u, cxp = (o.cross & 2u) != 0u;
    // the x-high face applies the outflow rule (it is the outflow face, and not a wall or
    // velocity face, whose rules win)
    const bool xout = OUTF && !(p.wall_mask & 2u) && !(p.vel_mask & 2u);
    xsel_load_f<OUTF, S, L>(pl, p, s, o, cxm, cxp, xout, f, std::make_integer_sequence<int, L::kQ>{});
    const bool gout = OUTF && cxp && p.heat_kind[1] == 3;
#pragma unroll
    for (int i = 0; i < kQT; ++i) {
        const int src = s + axis_off(ex7(i), o.xm, o.xp) + axis_off(ey7(i), o.ym, o.yp) +
                        axis_off(ez7(i), o.zm, o.zp);
        if (ex7(i) == 0) {
            g[i] = ldg_dev<S>(pl, p, i, src);
        } else {
            const bool bounce = ex7(i) == 1 ? cxm : (cxp && !gout);
            g[i] = ldg_either<S>(pl, p, i, opp7(i), bounce, bounce ? s : src);
        }
    }
    float hf[kOutSlots];
    if constexpr (OUTF) {
        const int yz = y + p.ny * z;
#pragma unroll
        for (int k = 0; k < kOutSlots; ++k) hf[k] = cxp ? __ldg(pl.hin + k * p.nyz + chk(yz, p.nyz)) : 0.0f;
    }
    if (!(cxm || cxp)) return;
    bool via[L::kQ];
    xsel_fix_f<OUTF, S, L>(p, cxm, cxp, xout, hf, f, via, std::make_integer_sequence<int, L::kQ>{});
    if (OUTF && cxp && xout) outflow_anchor<L>(f, via);
    if (cxm && p.heat_kind[0] == 2) g[1] = -g[1] + p.heat_abb[0];
    if (cxp) {
        if (gout) g[2] = outflow_blend(p, hf[5], g[2]);
        else if (p.heat_kind[1] == 2) g[2] = -g[2] + p.heat_abb[1];
    }
}

// How the sites of a warp gather: kGatherInterior when no pull of any of its sites crosses a
// non-periodic face, kGatherX when only x faces are crossed (the y and z neighbours of every
// site need no rule), else kGatherAny.  Warp-uniform: the caller votes (warp_gather_mode).
enum { kGatherInterior = 0, kGatherX = 1, kGatherAny = 2 };
__device__ __forceinline__ int warp_gather_mode(const KParams& p, int x, int y, int z, bool active) {
    if (__all_sync(0xffffffffu, !active || site_no_cross(p, x, y, z))) return kGatherInterior;
    if (__all_sync(0xffffffffu, !active || yz_fast(p, y, z))) return kGatherX;
    return kGatherAny;
}

// Pull of one site in the gather mode of its warp.
template <bool OUTF, class S, class L = D3Q19>
__device__ __forceinline__ void gather_site(const Planes& pl, const KParams& p, int x, int y, int z,
                                            int s, int mode, float* f, float* g) {
    if (mode == kGatherInterior) gather_interior<S, L>(pl, p, x, y, z, s, f, g);
    else if (mode == kGatherX) gather_xsel<OUTF, S, L>(pl, p, x, y, z, s, f, g);
    else gather_sel<OUTF, S, L>(pl, p, x, y, z, s, f, g);
}

// Outflow history, collision and store of one gathered site.
template <bool HET, bool OUTF, class S, bool ENTH = false, class L = D3Q19>
__device__ __forceinline__ void finish_site(const Planes& pl, const KParams& p, int x, int y, int z,
                                            int s, float* f, float* g) {
    if (OUTF && x == p.nx - 1) {
        const int yz = y + p.ny * z;
        pl.hout[0 * p.nyz + chk(yz, p.nyz)] = f[2];
        pl.hout[1 * p.nyz + chk(yz, p.nyz)] = f[8];
        pl.hout[2 * p.nyz + chk(yz, p.nyz)] = f[10];
        pl.hout[3 * p.nyz + chk(yz, p.nyz)] = f[12];
        pl.hout[4 * p.nyz + chk(yz, p.nyz)] = f[14];
        pl.hout[5 * p.nyz + chk(yz, p.nyz)] = g[2];
    }
    const Medium md = medium_at<HET>(p, s);
    collide_on<true, ENTH, L>(p, md, f, g, 0.0f, 0.0f, 0.0f, [&](const L1* gg, L1 dT) {
#pragma unroll
        for (int i = 0; i < kQT; ++i) stg_dev<S>(pl, p, i, s, gg[i].v, dT.v);
        if constexpr (S::kScaled) pl.tout[chk(s, p.ns)] = dT.v;
    });
#pragma unroll
    for (int i = 0; i < L::kQ; ++i) stp<S>(pl, p, i, s, f[i]);
}

// Programmatic dependent launch: a step kernel launched with it may be scheduled while the
// previous kernel of the stream drains.  Each thread first waits until that kernel has
// completed and its writes are visible (a no-op for an ordinary launch), then allows the next
// step's grid to be scheduled in turn.
// Block indices of a step kernel in its sweep order.  Blocks start roughly in launch order;
// lbm_step sets KParams::reverse on every other step, so that a step begins with the blocks
// whose inputs the previous step wrote last, many of them still in L2 (one FP32 population
// copy of the 256 x 64 x 64 channel is 109 MB against 126 MB of L2).  Measured on that
// channel: FP32 30.0k -> 32.8k MLUPS, FP16 37.8k -> 39.7k; 256^3 lattices gain under 1 %.
// Every block still runs once, reads only the copy being read and writes only the other:
// the order changes no result.
__device__ __forceinline__ int sweep_block(int b, int n, int reverse) {
    return reverse ? n - 1 - b : b;
}
__device__ __forceinline__ void dependent_launch_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// 3D launch: threadIdx.x + blockIdx.x * blockDim.x -> x, the same for y, blockIdx.z -> z.
// blockDim.x is the smallest power of two >= nx up to the block size (block_x_of): a warp
// holds one or more whole rows, or part of one, and votes as a whole over its lanes' sites.
// Registers: 64 per thread (32 resident warps per SM with 64-thread blocks); 72 with a porosity
// field, whose medium terms need more (28 warps; at 80 the field kernel lost 4 % on the 256^3
// cavity).
template <bool HET, bool OUTF, class S, bool ENTH = false, class L = D3Q19, bool NEE = false>
__global__ void __maxnreg__(HET ? 72 : 64)
    step_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl) {
    dependent_launch_prologue();
    const int x = sweep_block(blockIdx.x, gridDim.x, p.reverse) * blockDim.x + threadIdx.x;
    const int y = sweep_block(blockIdx.y, gridDim.y, p.reverse) * blockDim.y + threadIdx.y;
    const int z = sweep_block(blockIdx.z, gridDim.z, p.reverse);
    const bool valid = x < p.nx && y < p.ny;
    const unsigned nb = (NEE && valid) ? nee_bits(p, x, y, z) : 0u;  // node-wall site
    const bool streams = valid && nb == 0u;
    const int mode = warp_gather_mode(p, x, y, z, streams);
    if (!valid) return;
    float f[L::kQ], g[kQT];
    const int s = x + p.nx * (y + p.ny * z);
    if constexpr (NEE) {
        if (nb) {
            nee_site<HET, true, S, L>(pl, p, x, y, z, s, nb, f, g);
#pragma unroll
            for (int i = 0; i < L::kQ; ++i) stp<S>(pl, p, i, s, f[i]);
#pragma unroll
            for (int i = 0; i < kQT; ++i) stg_dev<S>(pl, p, i, s, g[i], 0.0f);
            return;
        }
    }
    gather_site<OUTF, S, L>(pl, p, x, y, z, s, mode, f, g);
    finish_site<HET, OUTF, S, ENTH, L>(pl, p, x, y, z, s, f, g);
}

// ---- paired sites: two x-adjacent sites per thread ----------------------------------------------
// One thread updates the sites x and x + 1 (x even, nx even) with the collision on L2 (the
// paired FP32 instructions).  A plane whose velocity has e_x = 0 holds the two sources next to
// each other, so it is read and written as one aligned 2-element access; the planes with
// e_x = +-1 read their two sources separately.  Warps with a boundary site gather each site on
// its own (gather_site) and pair the results.  The update is that of step_kernel, bit for bit.
template <class S>
__device__ __forceinline__ float2 ld2_raw(const typename S::T* a) {
    if constexpr (std::is_same<typename S::T, float>::value) {
        return __ldg(reinterpret_cast<const float2*>(a));
    } else if constexpr (std::is_same<typename S::T, __half>::value) {
        return __half22float2(__ldg(reinterpret_cast<const __half2*>(a)));
    } else {
        return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(a)));
    }
}
template <class S>
__device__ __forceinline__ void st2_raw(typename S::T* a, float2 v) {
    if constexpr (std::is_same<typename S::T, float>::value) {
        *reinterpret_cast<float2*>(a) = v;
    } else if constexpr (std::is_same<typename S::T, __half>::value) {
        *reinterpret_cast<__half2*>(a) = __float22half2_rn(v);
    } else {
        *reinterpret_cast<__nv_bfloat162*>(a) = __float22bfloat162_rn(v);
    }
}
// Plane q (flow) at the aligned pair idx, idx + 1, as ldp reads each.
template <class S>
__device__ __forceinline__ L2 ldp2(const Planes& pl, const KParams& p, int q, int idx) {
    idx = chk(idx + 1, p.ns) - 1;  // both elements of the pair in range
    return L2{ld2_raw<S>(at_in<S>(pl, p, q, idx))};
}
// D3Q7 population i at the aligned pair idx, idx + 1, as ldg_dev reads each.
template <class S>
__device__ __forceinline__ L2 ldg2(const Planes& pl, const KParams& p, int i, int idx) {
    if constexpr (!S::kScaled) {
        return ldp2<S>(pl, p, kQ + i, idx);
    } else {
        idx = chk(idx + 1, p.ns) - 1;
        const L2 st{ld2_raw<S>(at_in<S>(pl, p, kQ + i, idx))};
        const L2 tin{__ldg(reinterpret_cast<const float2*>(pl.tin + chk(idx, p.ns - 1)))};
        return K<L2>(i == 0 ? p.om0 : p.om1) * fma(K<L2>(p.sigma), tin, st);
    }
}
template <class S>
__device__ __forceinline__ void stp2(const Planes& pl, const KParams& p, int q, int idx, L2 v) {
    idx = chk(idx + 1, p.ns) - 1;
    st2_raw<S>(at_out<S>(pl, p, q, idx), v.v);
}
template <class S>
__device__ __forceinline__ void stg2(const Planes& pl, const KParams& p, int i, int idx, L2 v, L2 dT) {
    idx = chk(idx + 1, p.ns) - 1;
    if constexpr (!S::kScaled) {
        stp2<S>(pl, p, kQ + i, idx, v);
    } else {
        const L2 w = fma(v, K<L2>(i == 0 ? p.iom0 : p.iom1), -(K<L2>(p.sigma) * dT));
        st2_raw<S>(at_out<S>(pl, p, kQ + i, idx), w.v);
    }
}
__device__ __forceinline__ L2 pair(float a, float b) { return {make_float2(a, b)}; }

// Plane q's values at elements idx + d and idx + d + 1, as ldp reads each, both addressed from
// element idx.
template <class S>
__device__ __forceinline__ L2 ldp2_rel(const Planes& pl, const KParams& p, int q, int idx, int d) {
    return pair(S::ld(at_in_rel<S>(pl, p, q, idx, d)), S::ld(at_in_rel<S>(pl, p, q, idx, d + 1)));
}
// D3Q7 population i of a 16-bit format from its stored pair st and the temperature deviations
// T of its two source sites, as ldg_dev decodes each.
template <class S>
__device__ __forceinline__ L2 g_decode(const KParams& p, int i, L2 st, L2 T) {
    return K<L2>(i == 0 ? p.om0 : p.om1) * fma(K<L2>(p.sigma), T, st);
}

// Pull of the pair when no pull of either site crosses a face and no x pull wraps (x_a > 0,
// x_a + 2 < nx; warp_pair_mode sends the other pairs to gather_pair_x): the two sources of a
// plane with e_x = +-1 are the elements next to the pair's own and share its address; the
// thermal pulls of a 16-bit format take their source temperatures from the pair's own
// temperature row and the elements beside it.
template <class S>
__device__ __forceinline__ void gather_pair_interior(const Planes& pl, const KParams& p, int xa,
                                                     int y, int z, int sa, L2* f, L2* g) {
    const AxisOff o = axis_offsets(p, xa, y, z);  // site a; site b differs only along +x
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int row = sa + axis_off(D3Q19::ey(i), o.ym, o.yp) + axis_off(D3Q19::ez(i), o.zm, o.zp);
        if (D3Q19::ex(i) == 0) f[i] = ldp2<S>(pl, p, i, row);
        else if (D3Q19::ex(i) == 1) f[i] = ldp2_rel<S>(pl, p, i, row, -1);  // sources x - 1
        else f[i] = ldp2_rel<S>(pl, p, i, row, 1);                          // sources x + 1
    }
    if constexpr (!S::kScaled) {
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
            const int row = sa + axis_off(ey7(i), o.ym, o.yp) + axis_off(ez7(i), o.zm, o.zp);
            if (ex7(i) == 0) g[i] = ldp2<S>(pl, p, kQ + i, row);
            else g[i] = ldp2_rel<S>(pl, p, kQ + i, row, ex7(i) == 1 ? -1 : 1);
        }
    } else {
        // temperatures: the pair's own (x_a, x_a + 1) and the sites beside it (x_a - 1, x_a + 2)
        const float* tr = pl.tin + chk(sa, p.ns - 1);
        const L2 Ts{__ldg(reinterpret_cast<const float2*>(tr))};
#ifdef LBM_BOUNDS_CHECK
        const float Tm = __ldg(pl.tin + chk(sa - 1, p.ns)), Tp = __ldg(pl.tin + chk(sa + 2, p.ns));
#else
        const float Tm = __ldg(tr - 1), Tp = __ldg(tr + 2);
#endif
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
            const int row = sa + axis_off(ey7(i), o.ym, o.yp) + axis_off(ez7(i), o.zm, o.zp);
            if (ex7(i) == 0) {
                const L2 st{ld2_raw<S>(at_in<S>(pl, p, kQ + i, chk(row + 1, p.ns) - 1))};
                const L2 T = i == 0 ? Ts
                                    : L2{__ldg(reinterpret_cast<const float2*>(pl.tin + chk(row, p.ns - 1)))};
                g[i] = g_decode<S>(p, i, st, T);
            } else {
                const int d = ex7(i) == 1 ? -1 : 1;
                const L2 st = pair(S::ld(at_in_rel<S>(pl, p, kQ + i, row, d)),
                                   S::ld(at_in_rel<S>(pl, p, kQ + i, row, d + 1)));
                g[i] = g_decode<S>(p, i, st, ex7(i) == 1 ? pair(Tm, Ts.v.x) : pair(Ts.v.y, Tp));
            }
        }
    }
}

// The x faces' rules of gather_pair_x: site a (lane .x) on the x-low face, site b (lane .y) on
// the x-high face, as xsel_fix_f and outflow_anchor apply them to a single site.
template <bool OUTF, int... I>
__device__ __forceinline__ void pair_x_fix_f(const KParams& p, bool cxm, bool cxp, bool xout,
                                             const float* hf, L2* f,
                                             std::integer_sequence<int, I...>) {
    const bool vlo = (p.vel_mask & 1u) && !(p.wall_mask & 1u);
    const bool vhi = (p.vel_mask & 2u) && !(p.wall_mask & 2u);
    bool via[kQ];
    (([&] {
         constexpr int ex = D3Q19::ex(I);
         via[I] = false;
         if constexpr (ex == 1) {
             if (cxm && vlo) f[I].v.x = bounce_moving<D3Q19, I>(p, 0, f[I].v.x);
         } else if constexpr (ex == -1) {
             if (cxp) {
                 if (xout) {
                     if constexpr (OUTF) {
                         f[I].v.y = outflow_blend(p, hf[D3Q19::slot(I)], f[I].v.y);
                         via[I] = true;
                     }
                 } else if (vhi) {
                     f[I].v.y = bounce_moving<D3Q19, I>(p, 1, f[I].v.y);
                 }
             }
         }
     }()),
     ...);
    if (OUTF && cxp && xout) {
        float fb[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) fb[i] = f[i].v.y;
        outflow_anchor<D3Q19>(fb, via);
#pragma unroll
        for (int i = 0; i < kQ; ++i) f[i].v.y = fb[i];
    }
}

// Pull of a pair whose rows need no y/z face rule (yz_fast) but whose site a may lie on the
// x-low face or site b on the x-high face: the planes with e_x = 0 stay paired, the shifted
// planes select per site as gather_xsel does, and the x faces' rules apply to the site on the
// face (the same operations on each site as gather_xsel).
template <bool OUTF, class S>
__device__ __forceinline__ void gather_pair_x(const Planes& pl, const KParams& p, int xa, int y,
                                              int z, int sa, L2* f, L2* g) {
    const AxisOff o = axis_offsets(p, xa, y, z);  // site a; site b differs only along +x
    const bool cxm = (o.cross & 1u) != 0u;        // site a on a non-periodic x-low face
    const int sb = sa + 1;
    bool cxp = false;                              // site b on a non-periodic x-high face
    int xpb = 1;
    if (xa + 1 == p.nx - 1) {
        if (p.per_mask & 2u) xpb = 1 - p.nx;
        else { xpb = 0; cxp = true; }
    }
    const bool xout = OUTF && !(p.wall_mask & 2u) && !(p.vel_mask & 2u);
    const bool bnc_b = cxp && !xout;  // site b's -x pulls bounce back
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int oyz = axis_off(D3Q19::ey(i), o.ym, o.yp) + axis_off(D3Q19::ez(i), o.zm, o.zp);
        if (D3Q19::ex(i) == 0) {
            f[i] = ldp2<S>(pl, p, i, sa + oyz);
        } else if (D3Q19::ex(i) == 1) {
            f[i] = pair(ldp_either<S>(pl, p, i, D3Q19::opp(i), cxm, cxm ? sa : sa + o.xm + oyz),
                        ldp<S>(pl, p, i, sa + oyz));
        } else {
            f[i] = pair(ldp<S>(pl, p, i, sa + 1 + oyz),
                        ldp_either<S>(pl, p, i, D3Q19::opp(i), bnc_b, bnc_b ? sb : sb + xpb + oyz));
        }
    }
    const bool gout = OUTF && cxp && p.heat_kind[1] == 3;
#pragma unroll
    for (int i = 0; i < kQT; ++i) {
        const int oyz = axis_off(ey7(i), o.ym, o.yp) + axis_off(ez7(i), o.zm, o.zp);
        if (ex7(i) == 0) {
            g[i] = ldg2<S>(pl, p, i, sa + oyz);
        } else if (ex7(i) == 1) {
            g[i] = pair(ldg_either<S>(pl, p, i, opp7(i), cxm, cxm ? sa : sa + o.xm + oyz),
                        ldg_dev<S>(pl, p, i, sa + oyz));
        } else {
            const bool bb = cxp && !gout;
            g[i] = pair(ldg_dev<S>(pl, p, i, sa + 1 + oyz),
                        ldg_either<S>(pl, p, i, opp7(i), bb, bb ? sb : sb + xpb + oyz));
        }
    }
    float hf[kOutSlots];
    if constexpr (OUTF) {
        const int yz = y + p.ny * z;
#pragma unroll
        for (int k = 0; k < kOutSlots; ++k) hf[k] = cxp ? __ldg(pl.hin + k * p.nyz + chk(yz, p.nyz)) : 0.0f;
    }
    if (!(cxm || cxp)) return;
    pair_x_fix_f<OUTF>(p, cxm, cxp, xout, hf, f, std::make_integer_sequence<int, kQ>{});
    if (cxm && p.heat_kind[0] == 2) g[1].v.x = -g[1].v.x + p.heat_abb[0];
    if (cxp) {
        if (gout) g[2].v.y = outflow_blend(p, hf[5], g[2].v.y);
        else if (p.heat_kind[1] == 2) g[2].v.y = -g[2].v.y + p.heat_abb[1];
    }
}

// The gather mode of a warp of pairs: interior when no pull of any lane crosses a face and no
// x pull wraps (x_a > 0, x_a + 2 < nx); x-select when every lane's y/z pulls need no rule
// (this includes the pairs at the ends of a periodic x axis); else the general select.
__device__ __forceinline__ int warp_pair_mode(const KParams& p, int xa, int y, int z, bool active) {
    const bool quiet = yz_fast(p, y, z) && xa > 0 && xa + 2 < p.nx;
    if (__all_sync(0xffffffffu, !active || quiet)) return kGatherInterior;
    if (__all_sync(0xffffffffu, !active || yz_fast(p, y, z))) return kGatherX;
    return kGatherAny;
}

// The update of the pair (xa, xa + 1) at row y, slab z in the gather mode of its warp.
template <bool HET, bool OUTF, class S>
__device__ __forceinline__ void pair_update(const Planes& pl, const KParams& p, int xa, int y,
                                            int z, int mode) {
    const int sa = xa + p.nx * (y + p.ny * z);
    L2 f[kQ], g[kQT];
    if (mode == kGatherInterior) {
        gather_pair_interior<S>(pl, p, xa, y, z, sa, f, g);
    } else if (mode == kGatherX) {
        gather_pair_x<OUTF, S>(pl, p, xa, y, z, sa, f, g);
    } else {
        float fa[kQ], ga[kQT], fb[kQ], gb[kQT];
        gather_site<OUTF, S>(pl, p, xa, y, z, sa, mode, fa, ga);
        gather_site<OUTF, S>(pl, p, xa + 1, y, z, sa + 1, mode, fb, gb);
#pragma unroll
        for (int i = 0; i < kQ; ++i) f[i] = pair(fa[i], fb[i]);
#pragma unroll
        for (int i = 0; i < kQT; ++i) g[i] = pair(ga[i], gb[i]);
    }
    if (OUTF && xa + 1 == p.nx - 1) {  // site b on the outflow face: its pre-collision pulls
        const int yz = y + p.ny * z;
        pl.hout[0 * p.nyz + chk(yz, p.nyz)] = f[2].v.y;
        pl.hout[1 * p.nyz + chk(yz, p.nyz)] = f[8].v.y;
        pl.hout[2 * p.nyz + chk(yz, p.nyz)] = f[10].v.y;
        pl.hout[3 * p.nyz + chk(yz, p.nyz)] = f[12].v.y;
        pl.hout[4 * p.nyz + chk(yz, p.nyz)] = f[14].v.y;
        pl.hout[5 * p.nyz + chk(yz, p.nyz)] = g[2].v.y;
    }
    const MediumT<L2> md = medium_pair<HET>(p, sa);
    collide_t<L2, true>(p, md, f, g, 0.0f, 0.0f, 0.0f, [&](const L2* gg, L2 dT) {
#pragma unroll
        for (int i = 0; i < kQT; ++i) stg2<S>(pl, p, i, sa, gg[i], dT);
        if constexpr (S::kScaled) *reinterpret_cast<float2*>(pl.tout + chk(sa + 1, p.ns) - 1) = dT.v;
    });
#pragma unroll
    for (int i = 0; i < kQ; ++i) stp2<S>(pl, p, i, sa, f[i]);
}

// Registers (measured on the 256x64x64 channel and the 256^3 field cavity, GB300): uncapped
// the kernel takes ~128 and runs 14 warps per SM, latency-bound; 96 (16-bit) and 104 (FP32)
// give 20 warps at little spilling for a uniform medium; with a porosity field the 16-bit
// instance is fastest at 112 and the FP32 one uncapped (it spills heavily below that).
template <bool HET, bool OUTF, class S>
__global__ void __maxnreg__(HET ? (S::kScaled ? 112 : 128) : (S::kScaled ? 96 : 104))
    step_pair_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl) {
    dependent_launch_prologue();
    const int xa = 2 * (sweep_block(blockIdx.x, gridDim.x, p.reverse) * blockDim.x + threadIdx.x);
    const int y = sweep_block(blockIdx.y, gridDim.y, p.reverse) * blockDim.y + threadIdx.y;
    const int z = sweep_block(blockIdx.z, gridDim.z, p.reverse);
    const bool valid = xa < p.nx && y < p.ny;  // nx even: x + 1 < nx as well
    const int mode = warp_pair_mode(p, xa, y, z, valid);
    if (valid) pair_update<HET, OUTF, S>(pl, p, xa, y, z, mode);
}

// ---- AA pattern: one population copy, updated in place (FP32, D3Q19, no outflow) ----------
// Two layouts of the single copy alternate.  W ("swapped"): physical plane opp(i) at x holds
// the post-collision f*_i(x), i.e. the ping-pong state with its planes permuted.  N
// ("streamed"): physical plane i at x holds the pre-collision f_i(x) that a pull would gather,
// except where the pull of i crosses a non-periodic face: there it holds the raw f*_opp(i)(x)
// and the face rule is applied when it is read.
//  pull step (W -> N): the ping-pong gather through a permuted plane table, the collision, and
//    a push of f*_j to plane j at x + e_j (plane opp(j) at x when x + e_j lies outside);
//  local step (N -> W): own-site loads (face rule on crossing directions), the collision, and
//    stores to plane opp(i) at x.
// A thread writes exactly the locations it reads, so both steps are race-free in one copy, and
// each gathers the same values as the ping-pong pull: the populations agree bit for bit.
struct StoreF32InPlace {  // FP32 loads through the coherent path: the copy is written in place
    using T = float;
    static constexpr bool kScaled = false;
    static constexpr bool kStrided = false;  // the plane tables are permuted
    static constexpr bool kOff32 = false;
    static __device__ __forceinline__ float ld(const T* q) { return *q; }
    static __device__ __forceinline__ void st(T* q, float v) { *q = v; }
};

template <int J>
__device__ __forceinline__ void aa_push_f(const Planes& pl, const Nbr& n, float v) {
    constexpr int I = opp19(J);  // f*_J leaves towards x + e_J, the pull source of opp(J)
    constexpr int ex = ex19(I), ey = ey19(I), ez = ez19(I);
    const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                        axis_cross(ez, n.cross, 16u, 32u);
    if (cr == 0u)
        static_cast<float*>(pl.out[J])[n.s + axis_off(ex, n.xm, n.xp) + axis_off(ey, n.ym, n.yp) +
                                        axis_off(ez, n.zm, n.zp)] = v;
    else
        static_cast<float*>(pl.out[I])[n.s] = v;
}
template <int J>
__device__ __forceinline__ void aa_push_g(const Planes& pl, const Nbr& n, float v) {
    constexpr int I = opp7(J);
    constexpr int ex = ex7(I), ey = ey7(I), ez = ez7(I);
    const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                        axis_cross(ez, n.cross, 16u, 32u);
    if (cr == 0u)
        static_cast<float*>(pl.out[kQ + J])[n.s + axis_off(ex, n.xm, n.xp) +
                                             axis_off(ey, n.ym, n.yp) + axis_off(ez, n.zm, n.zp)] = v;
    else
        static_cast<float*>(pl.out[kQ + I])[n.s] = v;
}
template <int... J>
__device__ __forceinline__ void aa_push_all(const Planes& pl, const Nbr& n, const float* f,
                                            const float* g, std::integer_sequence<int, J...>) {
    (aa_push_f<J>(pl, n, f[J]), ...);
    ((J < kQT ? aa_push_g<(J < kQT ? J : 0)>(pl, n, g[J < kQT ? J : 0]) : void()), ...);
}

// Local-step read of f_I at site n: plane I at x; on a crossing direction plane I holds the
// raw f*_opp(I)(x), to which the ping-pong face rule is applied (pull_f through the permuted
// table `pw`, whose logical plane opp(I) is physical plane I).
template <int I>
__device__ __forceinline__ float aa_local_f(const Planes& pl, const Planes& pw, const KParams& p,
                                            const Nbr& n) {
    constexpr int ex = ex19(I), ey = ey19(I), ez = ez19(I);
    const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                        axis_cross(ez, n.cross, 16u, 32u);
    bool via = false;
    if (cr == 0u) return ldp<StoreF32InPlace>(pl, p, I, n.s);
    return pull_f<D3Q19, I, false, StoreF32InPlace>(pw, p, n, &via);
}
template <int I>
__device__ __forceinline__ float aa_local_g(const Planes& pl, const Planes& pw, const KParams& p,
                                            const Nbr& n) {
    constexpr int ex = ex7(I), ey = ey7(I), ez = ez7(I);
    const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                        axis_cross(ez, n.cross, 16u, 32u);
    if (cr == 0u) return ldp<StoreF32InPlace>(pl, p, kQ + I, n.s);
    return pull_g<I, false, StoreF32InPlace>(pw, p, n);
}
template <int... I>
__device__ __forceinline__ void aa_local_all(const Planes& pl, const Planes& pw, const KParams& p,
                                             const Nbr& n, float* f, float* g,
                                             std::integer_sequence<int, I...>) {
    ((f[I] = aa_local_f<I>(pl, pw, p, n)), ...);
    ((I < kQT ? (void)(g[I < kQT ? I : 0] = aa_local_g<(I < kQT ? I : 0)>(pl, pw, p, n)) : void()),
     ...);
}

// Pull-step update of one valid site (W -> N): pl.in is the permuted table (logical q at
// physical opp(q)), pl.out the identity table of the same copy; mode as in step_kernel.
template <bool HET>
__device__ __forceinline__ void aa_pull_site(const KParams& p, const Planes& pl, int x, int y,
                                             int z, int mode) {
    float f[kQ], g[kQT];
    const int s = x + p.nx * (y + p.ny * z);
    gather_site<false, StoreF32InPlace, D3Q19>(pl, p, x, y, z, s, mode, f, g);
    const Medium md = medium_at<HET>(p, s);
    collide_on<true, false, D3Q19>(p, md, f, g);
    const Nbr n = neighbourhood(p, x, y, z);
    aa_push_all(pl, n, f, g, std::make_integer_sequence<int, kQ>{});
}

// Local-step update of one valid site (N -> W): pl = (in: identity, out: permuted), pw = the
// permuted table as input.
template <bool HET>
__device__ __forceinline__ void aa_local_site(const KParams& p, const Planes& pl, const Planes& pw,
                                              int x, int y, int z) {
    float f[kQ], g[kQT];
    const Nbr n = neighbourhood(p, x, y, z);
    if (n.cross == 0u) {
#pragma unroll
        for (int i = 0; i < kQ; ++i) f[i] = ldp<StoreF32InPlace>(pl, p, i, n.s);
#pragma unroll
        for (int i = 0; i < kQT; ++i) g[i] = ldp<StoreF32InPlace>(pl, p, kQ + i, n.s);
    } else {
        aa_local_all(pl, pw, p, n, f, g, std::make_integer_sequence<int, kQ>{});
    }
    const Medium md = medium_at<HET>(p, n.s);
    collide_on<true, false, D3Q19>(p, md, f, g);
#pragma unroll
    for (int i = 0; i < kQ; ++i) stp<StoreF32InPlace>(pl, p, i, n.s, f[i]);
#pragma unroll
    for (int i = 0; i < kQT; ++i) stp<StoreF32InPlace>(pl, p, kQ + i, n.s, g[i]);
}

// Pull step over one lattice (3D launch as step_kernel).
template <bool HET>
__global__ void __launch_bounds__(kBlock, HET ? kStepMinBlocks - 1 : kStepMinBlocks)
    aa_pull_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl) {
    dependent_launch_prologue();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool valid = x < p.nx && y < p.ny;
    const int mode = warp_gather_mode(p, x, y, z, valid);
    if (valid) aa_pull_site<HET>(p, pl, x, y, z, mode);
}

// Local step over one lattice.
template <bool HET>
__global__ void __launch_bounds__(kBlock, HET ? kStepMinBlocks - 1 : kStepMinBlocks)
    aa_local_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                    const __grid_constant__ Planes pw) {
    dependent_launch_prologue();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x < p.nx && y < p.ny) aa_local_site<HET>(p, pl, pw, x, y, z);
}

// N -> W without a collision: f*_j(x) sits in plane j at x + e_j (N) and belongs in plane
// opp(j) at x (W), while f*_opp(j)(x + e_j) sits in the latter and belongs in the former, so
// the two are swapped; each pair is swapped once, by the site x of its direction j < opp(j).
// Crossing directions already hold the raw value where W wants it.  Pure data movement.
// pl.out: the identity plane table of the copy.
template <int J>
__device__ __forceinline__ void aa_swap_f(const Planes& pl, const Nbr& n) {
    if constexpr (J < opp19(J)) {
        constexpr int I = opp19(J);
        constexpr int ex = ex19(I), ey = ey19(I), ez = ez19(I);
        const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                            axis_cross(ez, n.cross, 16u, 32u);
        if (cr == 0u) {
            float* a = static_cast<float*>(pl.out[J]) + n.s + axis_off(ex, n.xm, n.xp) +
                       axis_off(ey, n.ym, n.yp) + axis_off(ez, n.zm, n.zp);
            float* b = static_cast<float*>(pl.out[I]) + n.s;
            const float va = *a, vb = *b;
            *a = vb;
            *b = va;
        }
    }
}
template <int J>
__device__ __forceinline__ void aa_swap_g(const Planes& pl, const Nbr& n) {
    if constexpr (J < opp7(J)) {
        constexpr int I = opp7(J);
        constexpr int ex = ex7(I), ey = ey7(I), ez = ez7(I);
        const unsigned cr = axis_cross(ex, n.cross, 1u, 2u) | axis_cross(ey, n.cross, 4u, 8u) |
                            axis_cross(ez, n.cross, 16u, 32u);
        if (cr == 0u) {
            float* a = static_cast<float*>(pl.out[kQ + J]) + n.s + axis_off(ex, n.xm, n.xp) +
                       axis_off(ey, n.ym, n.yp) + axis_off(ez, n.zm, n.zp);
            float* b = static_cast<float*>(pl.out[kQ + I]) + n.s;
            const float va = *a, vb = *b;
            *a = vb;
            *b = va;
        }
    }
}
template <int... J>
__device__ __forceinline__ void aa_swap_all(const Planes& pl, const Nbr& n,
                                            std::integer_sequence<int, J...>) {
    (aa_swap_f<J>(pl, n), ...);
    ((J < kQT ? aa_swap_g<(J < kQT ? J : 0)>(pl, n) : void()), ...);
}

__global__ void __launch_bounds__(kBlock) aa_normalize_kernel(const __grid_constant__ KParams p,
                                                              const __grid_constant__ Planes pl) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Nbr n = neighbourhood(p, x, y, z);
    aa_swap_all(pl, n, std::make_integer_sequence<int, kQ>{});
}

// Batched step: one flat grid over the blocks of many lattices.  blk_lat[b] names the lattice
// of block b; the lattice's parameters and planes are read in place through the read-only
// cache (uniform over the block).  A block covers `rows` consecutive z-planes of one
// (x-segment, y-band) column, so the lookup is paid once per `rows` site updates.  L and NEE
// as in step_kernel: the D3Q15 flow lattice, node walls (a node-wall site takes nee_site).
template <bool HET, bool OUTF, class S, bool ENTH = false, class L = D3Q19, bool NEE = false>
__global__ void __launch_bounds__(kBlock, kStepMinBlocks - 1)
    batch_step_kernel(const BatchLattice* __restrict__ tab,
                      const unsigned short* __restrict__ blk_lat, int flip, int rows) {
    const BatchLattice* B = tab + __ldg(blk_lat + blockIdx.x);
    const KParams& p = B->p;
    const Planes& pl = B->pl[B->cur ^ flip];
    const int bx = B->bx, gx = B->gx, gy = B->gy;
    const int local = (int)blockIdx.x - B->block_begin;
    const int by = blockDim.x / bx;
    const int tx = threadIdx.x & (bx - 1), ty = threadIdx.x / bx;
    const int bxi = local % gx, rest = local / gx;
    const int x = bxi * bx + tx;
    const int y = (rest % gy) * by + ty;
    const int z0 = (rest / gy) * rows;
    const bool valid = x < p.nx && y < p.ny;
    for (int r = 0; r < rows; ++r) {
        const int z = z0 + r;
        if (z >= p.nz) break;  // uniform over the block
        const unsigned nb = (NEE && valid) ? nee_bits(p, x, y, z) : 0u;  // node-wall site
        // every lane of the warp reaches the votes; only the valid lanes update a site (the
        // site update itself holds no warp-wide vote)
        const int mode = warp_gather_mode(p, x, y, z, valid && nb == 0u);
        if (!valid) continue;
        float f[L::kQ], g[kQT];
        const int s = x + p.nx * (y + p.ny * z);
        if constexpr (NEE) {
            if (nb) {
                nee_site<HET, true, S, L>(pl, p, x, y, z, s, nb, f, g);
#pragma unroll
                for (int i = 0; i < L::kQ; ++i) stp<S>(pl, p, i, s, f[i]);
#pragma unroll
                for (int i = 0; i < kQT; ++i) stg_dev<S>(pl, p, i, s, g[i], 0.0f);
                continue;
            }
        }
        gather_site<OUTF, S, L>(pl, p, x, y, z, s, mode, f, g);
        finish_site<HET, OUTF, S, ENTH, L>(pl, p, x, y, z, s, f, g);
    }
}

// Batched step with two x-adjacent sites per thread: the lattices of a group that the paired
// kernel takes (D3Q19, even nx, no node walls, no enthalpy model, 32-bit plane offsets).  The
// block -> pair mapping is that of batch_step_kernel over nx / 2 pairs per row; each pair is
// updated by pair_update, as step_pair_kernel updates it, bit for bit.  Its parameters come
// from the lattice table in global memory, not from the constant bank, and take registers of
// their own: 128 per thread (16 warps per SM) keeps its spills to a few bytes (at the single
// kernel's 96-104 it spilled 200-400 bytes).
template <bool HET, bool OUTF, class S>
__global__ void __maxnreg__(128)
    batch_pair_kernel(const BatchLattice* __restrict__ tab,
                      const unsigned short* __restrict__ blk_lat, int flip, int rows) {
    const BatchLattice* L = tab + __ldg(blk_lat + blockIdx.x);
    const KParams& p = L->p;
    const Planes& pl = L->pl[L->cur ^ flip];
    const int bx = L->bx, gx = L->gx, gy = L->gy;
    const int local = (int)blockIdx.x - L->block_begin;
    const int by = blockDim.x / bx;
    const int tx = threadIdx.x & (bx - 1), ty = threadIdx.x / bx;
    const int bxi = local % gx, rest = local / gx;
    const int xa = 2 * (bxi * bx + tx);
    const int y = (rest % gy) * by + ty;
    const int z0 = (rest / gy) * rows;
    const bool valid = xa < p.nx && y < p.ny;
    for (int r = 0; r < rows; ++r) {
        const int z = z0 + r;
        if (z >= p.nz) break;  // uniform over the block
        const int mode = warp_pair_mode(p, xa, y, z, valid);
        if (valid) pair_update<HET, OUTF, S>(pl, p, xa, y, z, mode);
    }
}

// Batched AA step: one flat grid over the blocks of the AA lattices of a group (FP32, D3Q19,
// no outflow), each lattice in its own phase.  Lattice L runs a pull step when
// (L->cur ^ flip) is 0 (its copy in the swapped layout) and a local step otherwise; L->pl[0] =
// (in: permuted, out: identity) and L->pl[1] = (in: identity, out: permuted) are the plane
// tables of its single copy, and pl[0] doubles as the local step's permuted input table.  The
// block -> site mapping is that of batch_step_kernel.
template <bool HET>
__global__ void __launch_bounds__(kBlock, kStepMinBlocks - 1)
    batch_aa_kernel(const BatchLattice* __restrict__ tab,
                    const unsigned short* __restrict__ blk_lat, int flip, int rows) {
    const BatchLattice* L = tab + __ldg(blk_lat + blockIdx.x);
    const KParams& p = L->p;
    const bool local = ((L->cur ^ flip) & 1) != 0;  // uniform over the block
    const int bx = L->bx, gx = L->gx, gy = L->gy;
    const int loc = (int)blockIdx.x - L->block_begin;
    const int by = blockDim.x / bx;
    const int tx = threadIdx.x & (bx - 1), ty = threadIdx.x / bx;
    const int bxi = loc % gx, rest = loc / gx;
    const int x = bxi * bx + tx;
    const int y = (rest % gy) * by + ty;
    const int z0 = (rest / gy) * rows;
    const bool valid = x < p.nx && y < p.ny;
    for (int r = 0; r < rows; ++r) {
        const int z = z0 + r;
        if (z >= p.nz) break;  // uniform over the block
        // every lane reaches the votes; only the valid lanes update a site
        const int mode = warp_gather_mode(p, x, y, z, valid);
        if (!valid) continue;
        if (local) aa_local_site<HET>(p, L->pl[1], L->pl[0], x, y, z);
        else aa_pull_site<HET>(p, L->pl[0], x, y, z, mode);
    }
}

template <bool HET, bool OUTF, class S, bool ENTH = false, class L = D3Q19, bool NEE = false>
__global__ void __launch_bounds__(kBlock)
    macros_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                  float* __restrict__ rho, float* __restrict__ u, float* __restrict__ T) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const Nbr n = neighbourhood(p, x, y, z);
    float f[L::kQ], g[kQT];
    Macro m;
    const unsigned nb = NEE ? nee_bits(p, x, y, z) : 0u;
    if (NEE && nb) {  // node-wall site: (rho_b, u_w, T_b)
        m = nee_site<HET, false, S, L>(pl, p, x, y, z, n.s, nb, f, g);
    } else {
        gather_general<OUTF, S, L>(pl, p, n, f, g);
        const Medium md = medium_at<HET>(p, n.s);
        m = collide_on<false, ENTH, L>(p, md, f, g);
    }
    const long long s = n.s;
    if (rho) rho[s] = m.rho;
    if (u) {
        u[s] = m.ux;
        u[p.ns + s] = m.uy;
        u[2 * p.ns + s] = m.uz;
    }
    if (T) T[s] = m.T;
}

// Equilibrium state (Eqs. 24 and 42) with rho = rho0, computed in FP64 and stored once
// rounded in the storage format (deviations, see the storage section above).
template <class S, class L = D3Q19>
__global__ void init_eq_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                               const double* __restrict__ T_field,
                               const double* __restrict__ u_field, double T_uniform) {
    long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.ns) return;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    if (u_field) {
        ux = u_field[s];
        uy = u_field[p.ns + s];
        uz = u_field[2 * p.ns + s];
    }
    double T = T_field ? T_field[s] : T_uniform;
    double phi = p.phi_field ? (double)p.phi_field[s] : (double)p.phi;
    double rho0 = p.rho0, usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < L::kQ; ++i) {
        double eu = L::ex(i) * ux + L::ey(i) * uy + L::ez(i) * uz;
        double w = L::wd(i);
        double rel = rho0 * (3.0 * eu + 4.5 * eu * eu / phi - 1.5 * usq / phi);  // dev / w
        S::st(static_cast<typename S::T*>(pl.out[i]) + s, (float)(S::kScaled ? kFlowUnit * w * rel : w * rel));
    }
    double varpi = p.varpi, sigma = p.sigma, T0 = p.T0, csT2 = varpi / 3.0;
    if (p.enthalpy) {
        // Eq. B12 with the phase-pure enthalpy of T (solid at or below T_s), full values
        const double En = T <= (double)p.ent_Ts ? T / (double)p.ent_is
                                                : (double)p.ent_El + (T - (double)p.ent_Tl) / (double)p.ent_il;
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
            const double eu = ex7(i) * ux + ey7(i) * uy + ez7(i) * uz;
            const double v = i == 0 ? En - varpi * p.c_ref * T
                                    : varpi * p.c_ref * T / 6.0 + 0.5 * eu * p.c_pl * T;
            S::st(static_cast<typename S::T*>(pl.out[kQ + i]) + s, (float)v);
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kQT; ++i) {
        double om = i == 0 ? 1.0 - varpi : varpi / 6.0;
        double eu = ex7(i) * ux + ey7(i) * uy + ez7(i) * uz;
        if (S::kScaled)  // (g_eq - omega sigma T) / omega
            S::st(static_cast<typename S::T*>(pl.out[kQ + i]) + s, (float)(T * eu / csT2));
        else  // g_eq - omega sigma T0
            S::st(static_cast<typename S::T*>(pl.out[kQ + i]) + s,
                  (float)(om * (sigma * (T - T0) + T * eu / csT2)));
    }
    if (S::kScaled) pl.tout[s] = (float)(T - T0);
}

// Host FP64 D3Q7 planes (full values, 7 x n) -> stored planes of a format with a temperature
// plane: T_x - T0 = sum_i g_i / sigma - T0, stored_i = g_i / omega_i - sigma T_x.
template <class S>
__global__ void g_to_dev_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                                const double* __restrict__ src, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double sum = 0.0;
#pragma unroll
        for (int i = 0; i < kQT; ++i) sum += src[i * n + k];
        const double T = sum / p.sigma;
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
            const double om = i == 0 ? (double)p.om0 : (double)p.om1;
            S::st(static_cast<typename S::T*>(pl.out[kQ + i]) + k,
                  (float)(src[i * n + k] / om - p.sigma * T));
        }
        pl.tout[k] = (float)(T - p.T0);
    }
}

// Stored D3Q7 planes of a format with a temperature plane -> host FP64 full values.
template <class S>
__global__ void g_to_host_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                                 double* __restrict__ dst, long long n) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double T = (double)pl.tin[k] + p.T0;
#pragma unroll
        for (int i = 0; i < kQT; ++i) {
            const double om = i == 0 ? (double)p.om0 : (double)p.om1;
            const double v = S::ld(static_cast<const typename S::T*>(pl.in[kQ + i]) + k);
            dst[i * n + k] = om * (v + p.sigma * T);
        }
    }
}

// Host FP64 population plane (full values) -> stored plane: (v - offset) / scale.
template <class S>
__global__ void plane_to_dev_kernel(const double* __restrict__ src, void* __restrict__ dst,
                                    double offset, double inv_scale, long long n) {
    typename S::T* d = static_cast<typename S::T*>(dst);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        S::st(d + k, (float)((src[k] - offset) * inv_scale));
}

// Stored plane -> FP64 full values: v * scale + offset.
template <class S>
__global__ void plane_to_host_kernel(const void* __restrict__ src, double* __restrict__ dst,
                                     double offset, double scale, long long n) {
    const typename S::T* q = static_cast<const typename S::T*>(src);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        dst[k] = (double)S::ld(q + k) * scale + offset;
}

template <class S>
__global__ void hist_reset_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                                  float* __restrict__ hist) {
    const int nyz = p.ny * p.nz;
    const int yz = blockIdx.x * blockDim.x + threadIdx.x;
    if (yz >= nyz) return;
    const int s = (p.nx - 1) + p.nx * yz;
    hist[0 * nyz + yz] = ldp<S>(pl, p, 2, s);
    hist[1 * nyz + yz] = ldp<S>(pl, p, 8, s);
    hist[2 * nyz + yz] = ldp<S>(pl, p, 10, s);
    hist[3 * nyz + yz] = ldp<S>(pl, p, 12, s);
    hist[4 * nyz + yz] = ldp<S>(pl, p, 14, s);
    hist[5 * nyz + yz] = ldg_dev<S>(pl, p, 2, s);
}

// ---- FP64 reductions ---------------------------------------------------------------------------
constexpr int kRedBlocks = 608;  // 4 per SM of a 152-SM GB300
constexpr int kRedThreads = 256;

template <int NV>
__device__ __forceinline__ void block_reduce_store(double (&v)[NV], double* out) {
    __shared__ double sh[NV][kRedThreads / 32];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = threadIdx.x < kRedThreads / 32 ? sh[k][threadIdx.x] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (threadIdx.x == 0) out[k] = x;
        }
    }
}

template <class S, class L = D3Q19>
__global__ void __launch_bounds__(kRedThreads)
    sums_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                double* __restrict__ partials) {
    double v[2] = {0.0, 0.0};
    for (int s = blockIdx.x * kRedThreads + threadIdx.x; s < p.ns; s += gridDim.x * kRedThreads) {
#pragma unroll
        for (int i = 0; i < L::kQ; ++i) v[0] += (double)ldp<S>(pl, p, i, s) * (double)p.inv_fu;
#pragma unroll
        for (int i = 0; i < kQT; ++i) v[1] += (double)ldg_dev<S>(pl, p, i, s);
    }
    block_reduce_store<2>(v, partials + 2 * blockIdx.x);
}

// Totals of nparts partial sums (NV values each) in a fixed order, by one block.
template <int NV>
__device__ __forceinline__ void finalize_sums(const double* __restrict__ partials, int nparts,
                                              double* __restrict__ out) {
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kRedThreads)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += partials[NV * b + k];
    block_reduce_store<NV>(v, out);
}
template <int NV>
__global__ void __launch_bounds__(kRedThreads)
    finalize_kernel(const double* __restrict__ partials, int nparts, double* __restrict__ out) {
    finalize_sums<NV>(partials, nparts, out);
}

// Residual sums of one site against the previous fields: v += (|u - u_prev|^2, |u|^2,
// (T - T_prev)^2, T^2, non-finite values).
__device__ __forceinline__ void residual_site(double (&v)[5], const float (&u)[3],
                                              const float (&up)[3], float T, float Tp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = u[a], d = x - (double)up[a];
        v[0] += d * d;
        v[1] += x * x;
        if (!isfinite(x)) v[4] += 1.0;
    }
    const double t = T, dt = t - (double)Tp;
    v[2] += dt * dt;
    v[3] += t * t;
    if (!isfinite(t)) v[4] += 1.0;
}

__global__ void __launch_bounds__(kRedThreads)
    residual_kernel(const float* __restrict__ u, const float* __restrict__ T,
                    const float* __restrict__ up, const float* __restrict__ Tp, long long ns,
                    double* __restrict__ partials) {
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long s = (long long)blockIdx.x * kRedThreads + threadIdx.x; s < ns;
         s += (long long)gridDim.x * kRedThreads) {
        const float uu[3] = {u[s], u[ns + s], u[2 * ns + s]};
        const float pu[3] = {up[s], up[ns + s], up[2 * ns + s]};
        residual_site(v, uu, pu, T[s], Tp[s]);
    }
    block_reduce_store<5>(v, partials + 5 * blockIdx.x);
}

// Batched residual (lbm_server): block b of the list takes lattice blk[b].x and, within it,
// the sites residual_kernel's block blk[b].y takes (the same stride over the same number of
// blocks), computes their macroscopic fields as macros_kernel does, stores them as the new
// snapshot and adds them up with residual_site: every lattice's partial sums are those of
// launch_macros + launch_residual, bit for bit.
template <bool HET, bool OUTF, class S, bool ENTH>
__global__ void __launch_bounds__(kRedThreads)
    batch_residual_kernel(const ResLattice* __restrict__ tab, const int2* __restrict__ blk) {
    const int2 lb = blk[blockIdx.x];
    const ResLattice& R = tab[lb.x];
    const KParams& p = R.p;
    const long long ns = p.ns, nxy = (long long)p.nx * p.ny;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long s = (long long)lb.y * kRedThreads + threadIdx.x; s < ns;
         s += (long long)R.nr * kRedThreads) {
        const int z = (int)(s / nxy), rem = (int)(s - (long long)z * nxy);
        const int y = rem / p.nx, x = rem - y * p.nx;
        const Nbr n = neighbourhood(p, x, y, z);
        float f[kQ], g[kQT];
        gather_general<OUTF, S, D3Q19>(R.pl, p, n, f, g);
        const Medium md = medium_at<HET>(p, n.s);
        const Macro m = collide_on<false, ENTH, D3Q19>(p, md, f, g);
        const float uu[3] = {m.ux, m.uy, m.uz};
        R.cu[s] = m.ux;
        R.cu[ns + s] = m.uy;
        R.cu[2 * ns + s] = m.uz;
        R.cT[s] = m.T;
        if (R.pu) {
            const float pu[3] = {R.pu[s], R.pu[ns + s], R.pu[2 * ns + s]};
            residual_site(v, uu, pu, m.T, R.pT[s]);
        } else {  // first residual: the fields against themselves
            residual_site(v, uu, uu, m.T, m.T);
        }
    }
    block_reduce_store<5>(v, R.partials + 5 * lb.y);
}

__global__ void __launch_bounds__(kRedThreads)
    batch_residual_finish_kernel(const ResLattice* __restrict__ tab) {
    const ResLattice& R = tab[blockIdx.x];
    finalize_sums<5>(R.partials, R.nr, R.out);
}

// Temperature at a site from the streamed D3Q7 populations (Eq. 39).
template <bool OUTF, class S>
__device__ __forceinline__ double temperature_at(const Planes& pl, const KParams& p, int x, int y,
                                                 int z) {
    if (const unsigned nb = nee_bits(p, x, y, z)) {
        // node-wall site: the wall temperature, or that of the fluid site beside it
        int c[3] = {x, y, z};
        for (int fc = 0; fc < 6; ++fc)
            if (nb & (1u << fc)) {
                if (p.heat_kind[fc] == 4) return (double)p.T0 + (double)p.face_dT[fc];
                c[fc >> 1] += (fc & 1) ? -1 : 1;
            }
        x = c[0];
        y = c[1];
        z = c[2];
    }
    const Nbr n = neighbourhood(p, x, y, z);
    float g[kQT];
    gather_g_bc<OUTF, S>(g, pl, p, n, std::make_integer_sequence<int, kQT>{});
    float n0 = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + g[6]);
    if (p.enthalpy) {  // Eq. B8
        float T, fl;
        enthalpy_state(p, n0, T, fl);
        return (double)T;
    }
    return (double)p.T0 + (double)n0 * (double)p.inv_sigma;
}

// One block per entry of the Nusselt profile (first tangential axis); threads average the
// local Nusselt number of Eq. 53 over the second tangential axis (Eq. 54).
template <bool OUTF, class S>
__global__ void __launch_bounds__(kRedThreads)
    nusselt_kernel(const __grid_constant__ KParams p, const __grid_constant__ Planes pl,
                   int face, double Tw, double scale, double* __restrict__ profile) {
    const int axis = face >> 1, hi = face & 1;
    const int n[3] = {p.nx, p.ny, p.nz};
    const int t1 = axis == 0 ? 1 : 0;            // profile axis
    const int t2 = axis == 2 ? 1 : 2;            // averaged axis
    const int j = blockIdx.x;
    double v[1] = {0.0};
    for (int k = threadIdx.x; k < n[t2]; k += kRedThreads) {
        int c0[3], c1[3];
        c0[t1] = c1[t1] = j;
        c0[t2] = c1[t2] = k;
        if (p.heat_kind[face] == 4) {  // node wall: the wall site, then two fluid sites
            c0[axis] = hi ? n[axis] - 2 : 1;
            c1[axis] = hi ? n[axis] - 3 : 2;
            double T1 = temperature_at<OUTF, S>(pl, p, c0[0], c0[1], c0[2]);
            double T2 = temperature_at<OUTF, S>(pl, p, c1[0], c1[1], c1[2]);
            v[0] += (3.0 * Tw - 4.0 * T1 + T2) / 2.0 * scale;
            continue;
        }
        c0[axis] = hi ? n[axis] - 1 : 0;
        c1[axis] = hi ? n[axis] - 2 : 1;
        double T0 = temperature_at<OUTF, S>(pl, p, c0[0], c0[1], c0[2]);
        double T1 = temperature_at<OUTF, S>(pl, p, c1[0], c1[1], c1[2]);
        v[0] += (8.0 * Tw - 9.0 * T0 + T1) / 3.0 * scale;
    }
    double out[1];
    __shared__ double res;
    block_reduce_store<1>(v, out);
    if (threadIdx.x == 0) res = out[0];
    __syncthreads();
    if (threadIdx.x == 0) profile[j] = res / n[t2];
}

// Nu_3D = mean of the profile (Eq. 55); Nu_mp = centre value (mean of the two middle entries
// for an even length).
__global__ void nusselt_finalize_kernel(const double* __restrict__ profile, int n,
                                        double* __restrict__ out) {
    double v[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += kRedThreads) v[0] += profile[j];
    double r[1];
    block_reduce_store<1>(v, r);
    if (threadIdx.x == 0) {
        out[0] = r[0] / n;
        out[1] = (n % 2 == 0) ? 0.5 * (profile[n / 2 - 1] + profile[n / 2]) : profile[n / 2];
    }
}

inline unsigned blocks_for(long long n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

// Block of p.block_threads (32..kBlock) threads: blockDim.x = the smallest power of two >= nx
// within that size, the rest along y.  A row narrower than a warp shares the warp with the
// next rows (a 16-wide lattice fills its warps instead of leaving half the lanes idle); the
// warp votes of the gathers test every lane's own site, so they hold for any rows.
int block_x_of(int nx, int nt) {
    int bx = 1;
    while (bx < nx && bx < nt) bx *= 2;
    return bx;
}

void site_grid(const KParams& p, dim3* grid, dim3* block) {
    int nt = p.block_threads >= 32 && p.block_threads <= kBlock ? p.block_threads : kBlock;
    int bx = block_x_of(p.nx, nt);
    int by = nt / bx > 0 ? nt / bx : 1;
    *block = dim3(bx, by, 1);
    *grid = dim3((p.nx + bx - 1) / bx, (p.ny + by - 1) / by, p.nz);
}

// Calls fn.template operator()<S>() with the storage traits of p.storage.
template <class Fn>
cudaError_t with_storage(int storage, Fn&& fn) {
    if (storage == 1) return fn(StoreF16{});
    if (storage == 2) return fn(StoreBF16{});
    return fn(StoreF32{});
}

}  // namespace

// The device code above is also compiled into the TMA translation unit (lbm_tma.cu), which
// defines LBM_DEVICE_ONLY to leave out the host launch wrappers below.
#ifndef LBM_DEVICE_ONLY
// ---- launch wrappers ---------------------------------------------------------------------------
int reduction_blocks() { return kRedBlocks; }
int residual_blocks(long long ns) {
    const long long b = (ns + 2047) / 2048;
    return b < 1 ? 1 : (b > kRedBlocks ? kRedBlocks : (int)b);
}

cudaError_t bounds_report(long long* first_bad, int* checked) {
#ifdef LBM_BOUNDS_CHECK
    *checked = 1;
    unsigned long long v = 0;
    const cudaError_t e = cudaMemcpyFromSymbol(&v, g_bounds_bad, sizeof(v));
    *first_bad = v ? (long long)(v - 1) : -1;
    return e;
#else
    *checked = 0;
    *first_bad = -1;
    return cudaSuccess;
#endif
}

int aa_swapped_plane(int q) { return q < kQ ? opp19(q) : kQ + opp7(q - kQ); }

int block_x(int nx, int block_threads) { return block_x_of(nx, block_threads); }

cudaError_t launch_batch_step(const BatchLattice* tab, const unsigned short* blk_lat, int nblocks,
                              int block_threads, int rows, int storage, bool het, bool outflow,
                              bool enthalpy, bool off32, bool pair, int qf, bool nee, int flip,
                              cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    if (nee) {  // node walls: FP32 storage, no outflow (validated on the host)
        auto k = qf == 15 ? (het ? batch_step_kernel<true, false, StoreF32, false, D3Q15, true>
                                 : batch_step_kernel<false, false, StoreF32, false, D3Q15, true>)
                          : (het ? batch_step_kernel<true, false, StoreF32, false, D3Q19, true>
                                 : batch_step_kernel<false, false, StoreF32, false, D3Q19, true>);
        k<<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        return cudaGetLastError();
    }
    if (qf == 15) {  // D3Q15 flow lattice: FP32 storage (validated on the host)
        auto k = het ? (outflow ? batch_step_kernel<true, true, StoreF32, false, D3Q15>
                                : batch_step_kernel<true, false, StoreF32, false, D3Q15>)
                     : (outflow ? batch_step_kernel<false, true, StoreF32, false, D3Q15>
                                : batch_step_kernel<false, false, StoreF32, false, D3Q15>);
        k<<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        return cudaGetLastError();
    }
    if (pair) {  // 32-bit plane offsets, no enthalpy model (pair_eligible)
        auto go = [&](auto tag) {
            using S = decltype(tag);
            auto k = het ? (outflow ? batch_pair_kernel<true, true, S> : batch_pair_kernel<true, false, S>)
                         : (outflow ? batch_pair_kernel<false, true, S> : batch_pair_kernel<false, false, S>);
            k<<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
            return cudaGetLastError();
        };
        if (storage == 1) return go(StoreF16o{});
        if (storage == 2) return go(StoreBF16o{});
        return go(StoreF32o{});
    }
    if (enthalpy) {
        batch_step_kernel<false, false, StoreF32, true>
            <<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        return cudaGetLastError();
    }
    auto pick = [&](auto&& fn) {
        if (!off32) return with_storage(storage, fn);
        if (storage == 1) return fn(StoreF16o{});
        if (storage == 2) return fn(StoreBF16o{});
        return fn(StoreF32o{});
    };
    return pick([&](auto tag) {
        using S = decltype(tag);
        if (het && outflow)
            batch_step_kernel<true, true, S><<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        else if (het)
            batch_step_kernel<true, false, S><<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        else if (outflow)
            batch_step_kernel<false, true, S><<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        else
            batch_step_kernel<false, false, S><<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
        return cudaGetLastError();
    });
}

cudaError_t launch_batch_aa(const BatchLattice* tab, const unsigned short* blk_lat, int nblocks,
                            int block_threads, int rows, bool het, int flip, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    if (het) batch_aa_kernel<true><<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
    else batch_aa_kernel<false><<<nblocks, block_threads, 0, st>>>(tab, blk_lat, flip, rows);
    return cudaGetLastError();
}

// Launch of a step kernel, with programmatic dependent launch when `pdl` is set.
template <class... KArgs, class... Args>
cudaError_t launch_kernel(bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

cudaError_t launch_step(const KParams& p, bool outflow, const Planes& pl, bool pdl,
                        cudaStream_t st) {
    dim3 grid, block;
    site_grid(p, &grid, &block);
    const bool het = p.phi_field != nullptr;
    if (p.enthalpy)  // FP32, uniform medium, no outflow (validated on the host)
        return launch_kernel(pdl, step_kernel<false, false, StoreF32, true>, grid, block, 0, st, p, pl);
    if (p.nee_mask) {  // node walls: FP32 storage, no outflow (validated on the host)
        auto k = p.qf == 15 ? (het ? step_kernel<true, false, StoreF32, false, D3Q15, true>
                                   : step_kernel<false, false, StoreF32, false, D3Q15, true>)
                            : (het ? step_kernel<true, false, StoreF32, false, D3Q19, true>
                                   : step_kernel<false, false, StoreF32, false, D3Q19, true>);
        return launch_kernel(pdl, k, grid, block, 0, st, p, pl);
    }
    if (p.qf == 15) {  // D3Q15 flow lattice: FP32 storage (validated on the host)
        auto k = het ? (outflow ? step_kernel<true, true, StoreF32, false, D3Q15>
                                : step_kernel<true, false, StoreF32, false, D3Q15>)
                     : (outflow ? step_kernel<false, true, StoreF32, false, D3Q15>
                                : step_kernel<false, false, StoreF32, false, D3Q15>);
        return launch_kernel(pdl, k, grid, block, 0, st, p, pl);
    }
    auto go = [&](auto tag) {
        using S = decltype(tag);
        auto k = het ? (outflow ? step_kernel<true, true, S> : step_kernel<true, false, S>)
                     : (outflow ? step_kernel<false, true, S> : step_kernel<false, false, S>);
        return launch_kernel(pdl, k, grid, block, 0, st, p, pl);
    };
    if (p.off32) {  // 32-bit plane offsets (every lattice below ~82 M sites)
        if (p.storage == 1) return go(StoreF16o{});
        if (p.storage == 2) return go(StoreBF16o{});
        return go(StoreF32o{});
    }
    return with_storage(p.storage, go);
}

cudaError_t launch_step_pair(const KParams& p, bool outflow, const Planes& pl, bool pdl,
                             cudaStream_t st) {
    int nt = p.block_threads >= 32 && p.block_threads <= kBlock ? p.block_threads : 64;
    const int npx = p.nx / 2;
    const int bx = block_x_of(npx, nt);
    const int by = nt / bx > 0 ? nt / bx : 1;
    const dim3 block(bx, by, 1), grid((npx + bx - 1) / bx, (p.ny + by - 1) / by, p.nz);
    const bool het = p.phi_field != nullptr;
    auto go = [&](auto tag) {
        using S = decltype(tag);
        auto k = het ? (outflow ? step_pair_kernel<true, true, S> : step_pair_kernel<true, false, S>)
                     : (outflow ? step_pair_kernel<false, true, S> : step_pair_kernel<false, false, S>);
        return launch_kernel(pdl, k, grid, block, 0, st, p, pl);
    };
    if (p.storage == 1) return go(StoreF16o{});
    if (p.storage == 2) return go(StoreBF16o{});
    return go(StoreF32o{});
}

cudaError_t launch_aa_step(const KParams& p, bool local, const Planes& pl, const Planes& pw,
                           bool pdl, cudaStream_t st) {
    dim3 grid, block;
    site_grid(p, &grid, &block);
    const bool het = p.phi_field != nullptr;
    if (local)
        return launch_kernel(pdl, het ? aa_local_kernel<true> : aa_local_kernel<false>, grid, block,
                             0, st, p, pl, pw);
    return launch_kernel(pdl, het ? aa_pull_kernel<true> : aa_pull_kernel<false>, grid, block, 0,
                         st, p, pl);
}

cudaError_t launch_aa_normalize(const KParams& p, const Planes& pl, cudaStream_t st) {
    dim3 grid, block;
    site_grid(p, &grid, &block);
    aa_normalize_kernel<<<grid, block, 0, st>>>(p, pl);
    return cudaGetLastError();
}

cudaError_t launch_macros(const KParams& p, bool outflow, const Planes& pl, float* rho, float* u,
                          float* T, cudaStream_t st) {
    dim3 grid, block;
    site_grid(p, &grid, &block);
    const bool het = p.phi_field != nullptr;
    if (p.enthalpy) {
        macros_kernel<false, false, StoreF32, true><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        return cudaGetLastError();
    }
    if (p.nee_mask) {
        if (p.qf == 15) {
            if (het)
                macros_kernel<true, false, StoreF32, false, D3Q15, true><<<grid, block, 0, st>>>(p, pl, rho, u, T);
            else
                macros_kernel<false, false, StoreF32, false, D3Q15, true><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        } else {
            if (het)
                macros_kernel<true, false, StoreF32, false, D3Q19, true><<<grid, block, 0, st>>>(p, pl, rho, u, T);
            else
                macros_kernel<false, false, StoreF32, false, D3Q19, true><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        }
        return cudaGetLastError();
    }
    if (p.qf == 15) {
        if (het && outflow)
            macros_kernel<true, true, StoreF32, false, D3Q15><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        else if (het)
            macros_kernel<true, false, StoreF32, false, D3Q15><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        else if (outflow)
            macros_kernel<false, true, StoreF32, false, D3Q15><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        else
            macros_kernel<false, false, StoreF32, false, D3Q15><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        return cudaGetLastError();
    }
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        if (het && outflow)
            macros_kernel<true, true, S><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        else if (het)
            macros_kernel<true, false, S><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        else if (outflow)
            macros_kernel<false, true, S><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        else
            macros_kernel<false, false, S><<<grid, block, 0, st>>>(p, pl, rho, u, T);
        return cudaGetLastError();
    });
}

cudaError_t launch_init_eq(const KParams& p, const Planes& pl, const double* T_field,
                           const double* u_field, double T_uniform, cudaStream_t st) {
    if (p.qf == 15) {
        init_eq_kernel<StoreF32, D3Q15><<<blocks_for(p.ns, 128), 128, 0, st>>>(p, pl, T_field, u_field,
                                                                              T_uniform);
        return cudaGetLastError();
    }
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        init_eq_kernel<S><<<blocks_for(p.ns, 128), 128, 0, st>>>(p, pl, T_field, u_field, T_uniform);
        return cudaGetLastError();
    });
}

cudaError_t launch_plane_to_dev(int storage, const double* src, void* dst, double offset,
                                double scale, long long n, cudaStream_t st) {
    return with_storage(storage, [&](auto tag) {
        using S = decltype(tag);
        plane_to_dev_kernel<S><<<1216, 256, 0, st>>>(src, dst, offset, 1.0 / scale, n);
        return cudaGetLastError();
    });
}

cudaError_t launch_plane_to_host(int storage, const void* src, double* dst, double offset,
                                 double scale, long long n, cudaStream_t st) {
    return with_storage(storage, [&](auto tag) {
        using S = decltype(tag);
        plane_to_host_kernel<S><<<1216, 256, 0, st>>>(src, dst, offset, scale, n);
        return cudaGetLastError();
    });
}

cudaError_t launch_g_to_dev(const KParams& p, const Planes& pl, const double* src, cudaStream_t st) {
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        g_to_dev_kernel<S><<<1216, 256, 0, st>>>(p, pl, src, p.ns);
        return cudaGetLastError();
    });
}

cudaError_t launch_g_to_host(const KParams& p, const Planes& pl, double* dst, cudaStream_t st) {
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        g_to_host_kernel<S><<<1216, 256, 0, st>>>(p, pl, dst, p.ns);
        return cudaGetLastError();
    });
}

cudaError_t launch_hist_reset(const KParams& p, const Planes& pl, float* hist, cudaStream_t st) {
    const long long nyz = (long long)p.ny * p.nz;
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        hist_reset_kernel<S><<<blocks_for(nyz, 128), 128, 0, st>>>(p, pl, hist);
        return cudaGetLastError();
    });
}

cudaError_t launch_sums(const KParams& p, const Planes& pl, double* partials, int nparts,
                        double* out, cudaStream_t st) {
    if (p.qf == 15) {
        sums_kernel<StoreF32, D3Q15><<<nparts, kRedThreads, 0, st>>>(p, pl, partials);
        finalize_kernel<2><<<1, kRedThreads, 0, st>>>(partials, nparts, out);
        return cudaGetLastError();
    }
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        sums_kernel<S><<<nparts, kRedThreads, 0, st>>>(p, pl, partials);
        finalize_kernel<2><<<1, kRedThreads, 0, st>>>(partials, nparts, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_nusselt(const KParams& p, bool outflow, const Planes& pl, int face, double Tw,
                           double scale, double* profile, double* out, cudaStream_t st) {
    const int axis = face >> 1;
    const int n1 = axis == 0 ? p.ny : p.nx;
    return with_storage(p.storage, [&](auto tag) {
        using S = decltype(tag);
        if (outflow)
            nusselt_kernel<true, S><<<n1, kRedThreads, 0, st>>>(p, pl, face, Tw, scale, profile);
        else
            nusselt_kernel<false, S><<<n1, kRedThreads, 0, st>>>(p, pl, face, Tw, scale, profile);
        nusselt_finalize_kernel<<<1, kRedThreads, 0, st>>>(profile, n1, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_batch_residual(const ResLattice* tab, const int2* blk, int nblocks, bool het,
                                  bool outflow, int storage, bool enthalpy, cudaStream_t st) {
    if (nblocks < 1) return cudaSuccess;
    if (enthalpy) {  // FP32, uniform medium, no outflow (the model's rules)
        batch_residual_kernel<false, false, StoreF32, true><<<nblocks, kRedThreads, 0, st>>>(tab, blk);
        return cudaGetLastError();
    }
    auto go = [&](auto tag) {
        using S = decltype(tag);
        auto k = het ? (outflow ? batch_residual_kernel<true, true, S, false>
                                : batch_residual_kernel<true, false, S, false>)
                     : (outflow ? batch_residual_kernel<false, true, S, false>
                                : batch_residual_kernel<false, false, S, false>);
        k<<<nblocks, kRedThreads, 0, st>>>(tab, blk);
        return cudaGetLastError();
    };
    return with_storage(storage, go);
}

cudaError_t launch_batch_residual_finish(const ResLattice* tab, int n, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    batch_residual_finish_kernel<<<n, kRedThreads, 0, st>>>(tab);
    return cudaGetLastError();
}

cudaError_t launch_residual(const float* u, const float* T, const float* up, const float* Tp,
                            long long ns, double* partials, int nparts, double* out,
                            cudaStream_t st) {
    residual_kernel<<<nparts, kRedThreads, 0, st>>>(u, T, up, Tp, ns, partials);
    finalize_kernel<5><<<1, kRedThreads, 0, st>>>(partials, nparts, out);
    return cudaGetLastError();
}

#endif  // LBM_DEVICE_ONLY

}  // namespace lbm
