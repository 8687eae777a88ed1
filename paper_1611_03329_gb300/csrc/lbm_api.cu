// Host side of the C ABI declared in include/lbm.h: parameter mapping (Sec. 2, Sec. 4),
// validation, device memory of a context and the launch sequence of each call.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>  // header-only; ranges reach a profiler only when one is attached

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

namespace {
// NVTX range for the lifetime of the object: the host calls that queue or wait for GPU work
// show up as named ranges on a profiler's timeline (no cost without a profiler).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

using lbm::KParams;

struct lbm_ctx {
    lbm_params prm;
    lbm_lattice lat;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long ns = 0, sq = 0, nyz = 0;
    void* pop[2] = {nullptr, nullptr};    // ping-pong population copies, 26 planes each
    size_t elem = sizeof(float);          // bytes per stored population value
    float* hist[2] = {nullptr, nullptr};  // outflow history, 6 x ny*nz
    float* tplane[2] = {nullptr, nullptr};  // T - T0 per site (16-bit formats only)
    int cur = 0;
    lbm::Planes pl[2];  // launch planes reading copy 0 / copy 1
    bool outflow = false;
    int block_threads = 64;      // site-kernel block size (lbm_set_launch)
    bool pdl = true;             // step launches as programmatic dependent launches (lbm_set_launch)
    // AA scheme: one copy (pop[0]); pl[0] = (in: permuted, out: identity) for pull steps and
    // readers, pl[1] = (in: identity, out: permuted) for local steps and the initial state,
    // pw.in = permuted; aa_phase 0: swapped layout (next step pulls), 1: streamed layout
    bool aa = false;
    lbm::Planes pw;
    int aa_phase = 0;
    float* phi_dev = nullptr;
    KParams kp{};
    double* partials = nullptr;  // reduction scratch
    double* profile = nullptr;   // Nusselt profile scratch
    double* dres = nullptr;      // small device results
    double* hres = nullptr;      // pinned host mirror of dres
    double* stage = nullptr;     // FP64 staging, 7 x ns doubles (lazy)
    float* mac = nullptr;        // macro scratch, 9 x ns floats (lazy): two halves of (u, T)
                                 // and one rho plane; half `snap` holds the residual snapshot
    int snap = 0;
    bool have_prev = false;
    long long steps = 0;
    lbm_status sticky = LBM_OK;
    char err[512] = {0};
    // step kernel (LBM_KERNEL_*): for LBM_KERNEL_TMA the tensor maps of either copy, the
    // persistent grid and the device flag of a staged load that timed out
    int step_kernel = LBM_KERNEL_PLAIN;
    lbm::TmaMaps tmaps[2];
    int tma_blocks = 0;
    int* tma_err = nullptr;
    int tma_extra_tx = 0;  // test hook: bytes each stage waits for beyond its loads
};

namespace {

constexpr double kCs2 = 1.0 / 3.0;  // c_s^2 with c = 1

lbm_status fail(lbm_ctx* c, lbm_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
        if (s == LBM_ECUDA || s == LBM_ENOMEM) c->sticky = s;
    }
    return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define LBM_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }
bool rate_ok(double s) { return std::isfinite(s) && s > 0.0 && s < 2.0; }

// Relaxation rates of Sec. 4 where the caller left a non-positive value.
double or_default(double v, double d) { return v > 0.0 ? v : d; }

// Eq. 56 / Eq. 51 / lattice units -> lbm_lattice (default medium).  Returns an error text or
// nullptr.
// Whether a problem can run the AA scheme (L: its lattice so far, with q and node_walls set).
bool aa_eligible(const lbm_params* p, const lbm_lattice& L) {
    return L.q == 19 && p->storage == LBM_STORE_FP32 && !L.node_walls && !p->enthalpy &&
           p->flow_bc[1] != LBM_FLOW_OUTFLOW;
}

unsigned long long footprint_of(const lbm_params* p, const lbm_lattice& L, int has_phi_field);

const char* derive(const lbm_params* p, lbm_lattice* L) {
    std::memset(L, 0, sizeof(*L));
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return "nx, ny, nz must be >= 1";
    double ns = (double)p->nx * p->ny * p->nz;
    if (ns >= 2147483647.0) return "lattice too large (sites must fit in 31 bits)";
    if (p->nz > 65535) return "nz must be <= 65535 (one grid slice per z-plane)";
    if (p->storage != LBM_STORE_FP32 && p->storage != LBM_STORE_FP16_DEV &&
        p->storage != LBM_STORE_BF16_DEV)
        return "unknown storage format";
    L->q = p->q_flow == 0 ? 19 : p->q_flow;
    if (L->q != 19 && L->q != 15) return "q_flow must be 19 (D3Q19) or 15 (D3Q15)";
    if (L->q == 15 && p->storage != LBM_STORE_FP32) return "D3Q15 runs with FP32 storage only";
    if (!finite_pos(p->rho0)) return "rho0 must be > 0";
    if (!(p->varpi > 0.0 && p->varpi < 1.0)) return "varpi must lie in (0, 1)";
    if (!finite_pos(p->sigma)) return "sigma must be > 0";
    if (!finite_pos(p->J)) return "J must be > 0";
    if (!finite_pos(p->Gamma)) return "Gamma must be > 0";
    if (!std::isfinite(p->T0)) return "T0 must be finite";
    double dT = p->dT > 0.0 ? p->dT : 1.0;
    L->nx = p->nx;
    L->ny = p->ny;
    L->nz = p->nz;
    L->rho0 = p->rho0;
    L->T0 = p->T0;
    L->sigma = p->sigma;
    L->varpi = p->varpi;
    L->dT = dT;
    double s_e = or_default(p->s_e, 1.1), s_eps = or_default(p->s_eps, 1.1);
    double s_q = or_default(p->s_q, 1.1), s_pi = or_default(p->s_pi, 1.1);
    double s_m = or_default(p->s_m, 1.2);
    L->zeta_T = or_default(p->zeta_T, 1.0);
    L->zeta_e = or_default(p->zeta_e, 1.2);
    L->zeta_nu = or_default(p->zeta_nu, 1.2);
    double inv_s_nu, Lc;
    if (p->mapping == LBM_MAP_CAVITY) {
        Lc = p->L > 0.0 ? p->L : p->nx;
        if (!finite_pos(p->Ra) || !finite_pos(p->Pr) || !finite_pos(p->Ma))
            return "cavity mapping needs Ra, Pr, Ma > 0";
        // Eq. 56: 1/s_nu = 1/2 + Ma J L sqrt(3 Pr) / (c dt sqrt(Ra))
        inv_s_nu = 0.5 + p->Ma * p->J * Lc * std::sqrt(3.0 * p->Pr) / std::sqrt(p->Ra);
        L->nu_e = kCs2 * (inv_s_nu - 0.5);  // Eq. 32
        L->nu = L->nu_e / p->J;             // J = nu_e / nu (Eq. 7)
        L->alpha_f = L->nu / p->Pr;         // Pr = nu / alpha (Eq. 7)
        double uc = p->Ma * std::sqrt(kCs2);  // u_c = Ma c_s = sqrt(g beta dT L)
        L->gbeta = uc * uc / (dT * Lc);
    } else if (p->mapping == LBM_MAP_CHANNEL) {
        Lc = p->L > 0.0 ? p->L : p->ny;
        if (!finite_pos(p->Re) || !finite_pos(p->u0) || !finite_pos(p->Pr))
            return "channel mapping needs Re, u0, Pr > 0";
        if (!(p->Ri >= 0.0) || !std::isfinite(p->Ri)) return "Ri must be >= 0";
        // Eq. 51 with 1/s_nu on the left: nu_e = c_s^2 (1/s_nu - 1/2) = J H u0 / Re
        inv_s_nu = 0.5 + p->J * Lc * p->u0 / (kCs2 * p->Re);
        L->nu_e = kCs2 * (inv_s_nu - 0.5);
        L->nu = L->nu_e / p->J;
        L->alpha_f = L->nu / p->Pr;
        L->gbeta = p->Ri * p->u0 * p->u0 / (dT * Lc);  // Ri = g beta dT H / u0^2
    } else if (p->mapping == LBM_MAP_LATTICE) {
        Lc = p->L > 0.0 ? p->L : p->nx;
        if (!finite_pos(p->nu_e)) return "lattice mapping needs nu_e > 0";
        inv_s_nu = 0.5 + p->nu_e / kCs2;
        L->nu_e = p->nu_e;
        L->nu = L->nu_e / p->J;
        if (p->alpha_f > 0.0) {
            L->alpha_f = p->alpha_f;
        } else {
            if (!finite_pos(p->Pr)) return "Pr must be > 0";
            L->alpha_f = L->nu / p->Pr;
        }
        if (!std::isfinite(p->gbeta)) return "gbeta must be finite";
        L->gbeta = p->gbeta;
    } else {
        return "unknown mapping";
    }
    L->L = Lc;
    L->s_nu = 1.0 / inv_s_nu;
    double sv[19] = {1.0,   s_e,    s_eps, 1.0,    s_q,    1.0,    s_q,    1.0,    s_q,   L->s_nu,
                     s_pi,  L->s_nu, s_pi, L->s_nu, L->s_nu, L->s_nu, s_m, s_m, s_m};
    std::memcpy(L->s, sv, sizeof(sv));
    for (int k = 0; k < 19; ++k)
        if (!rate_ok(L->s[k])) return "a D3Q19 relaxation rate lies outside (0, 2)";
    if (!rate_ok(L->zeta_T) || !rate_ok(L->zeta_e) || !rate_ok(L->zeta_nu))
        return "a D3Q7 relaxation rate lies outside (0, 2)";
    L->Gamma = p->Gamma;
    L->alpha_m = -1.0;
    double csT2 = p->varpi / 3.0;
    L->zeta_alpha = 1.0 / (0.5 + p->Gamma * L->alpha_f / (p->sigma * csT2));  // Eq. 41
    if (!rate_ok(L->zeta_alpha)) return "zeta_alpha lies outside (0, 2)";
    if (p->gravity_axis < 0 || p->gravity_axis > 2) return "gravity_axis must be 0, 1 or 2";
    if (p->gravity_sign != 1 && p->gravity_sign != -1) return "gravity_sign must be +-1";
    for (int a = 0; a < 3; ++a) {
        L->buoy[a] = 0.0;
        if (!std::isfinite(p->accel[a])) return "accel must be finite";
        L->accel[a] = p->accel[a];
    }
    // G = -g beta (T - T0) with g pointing along gravity_sign * axis (Eq. 5)
    L->buoy[p->gravity_axis] = -(double)p->gravity_sign * L->gbeta;
    L->phi = 1.0;
    L->K = p->Da > 0.0 ? p->Da * Lc * Lc : HUGE_VAL;  // Da = K / L^2 (Eq. 7)
    L->F_phi = 0.0;
    L->phi_ref = 1.0;
    L->has_phi_field = 0;
    L->U_out = p->U_out > 0.0 ? p->U_out : p->u0;

    // boundaries
    int n[3] = {p->nx, p->ny, p->nz};
    for (int f = 0; f < 6; ++f) {
        int fk = p->flow_bc[f], hk = p->heat_bc[f];
        if (fk < 0 || fk > 4 || hk < 0 || hk > 5) return "unknown boundary kind";
        if ((fk == LBM_FLOW_NEE) != (hk == LBM_HEAT_NEE_DIRICHLET || hk == LBM_HEAT_NEE_ADIABATIC))
            return "a node wall (non-equilibrium extrapolation) is one for both flow and heat";
        if (fk == LBM_FLOW_NEE && n[f >> 1] < 3) return "a node wall needs >= 3 sites normal to it";
        if ((fk == LBM_FLOW_PERIODIC) != (hk == LBM_HEAT_PERIODIC))
            return "a face must be periodic for both flow and heat, or for neither";
        int other = f ^ 1;
        if ((fk == LBM_FLOW_PERIODIC) != (p->flow_bc[other] == LBM_FLOW_PERIODIC))
            return "periodic faces come in pairs";
        if (fk == LBM_FLOW_OUTFLOW && f != 1) return "outflow only on the x-high face";
        if (hk == LBM_HEAT_OUTFLOW && fk != LBM_FLOW_OUTFLOW)
            return "thermal outflow needs a flow outflow face";
        if ((hk == LBM_HEAT_DIRICHLET || hk == LBM_HEAT_NEE_DIRICHLET) && !std::isfinite(p->face_T[f]))
            return "face temperature must be finite";
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(p->face_u[f][a])) return "face velocity must be finite";
    }
    bool nee = false;
    for (int f = 0; f < 6; ++f) nee = nee || p->flow_bc[f] == LBM_FLOW_NEE;
    if (nee && p->flow_bc[1] == LBM_FLOW_OUTFLOW) return "node walls and an outflow do not mix";
    if (nee && p->storage != LBM_STORE_FP32) return "node walls run with FP32 storage only";
    if (nee && p->enthalpy) return "node walls do not run the enthalpy model";
    L->node_walls = nee ? 1 : 0;
    if (p->flow_bc[1] == LBM_FLOW_OUTFLOW) {
        if (n[0] < 3) return "an outflow needs nx >= 3";
        if (!finite_pos(L->U_out)) return "outflow speed must be > 0";
    }
    if (p->scheme < LBM_SCHEME_PINGPONG || p->scheme > LBM_SCHEME_AUTO)
        return "scheme must be LBM_SCHEME_PINGPONG, LBM_SCHEME_AA or LBM_SCHEME_AUTO";
    if (p->scheme == LBM_SCHEME_AA && !aa_eligible(p, *L))
        return "the AA scheme needs FP32 storage, D3Q19, no outflow, no node walls and no "
               "enthalpy model";
    // AUTO resolves to ping-pong here; lbm_create switches it to AA when two copies do not fit
    L->scheme = p->scheme == LBM_SCHEME_AA ? LBM_SCHEME_AA : LBM_SCHEME_PINGPONG;
    if (!std::isfinite(p->T_init)) return "T_init must be finite";
    L->enthalpy = p->enthalpy ? 1 : 0;
    L->flow_off = p->flow_off ? 1 : 0;
    if (p->enthalpy) {
        if (p->storage != LBM_STORE_FP32) return "the enthalpy model stores FP32 populations";
        if (p->flow_bc[1] == LBM_FLOW_OUTFLOW) return "the enthalpy model has no outflow";
        if (L->q == 15) return "the enthalpy model runs on the D3Q19 lattice";
        if (!finite_pos(p->St) || !finite_pos(p->c_pl) || !finite_pos(p->c_ps) ||
            !finite_pos(p->alpha_ratio))
            return "St, c_pl, c_ps and alpha_ratio must be > 0";
        if (!std::isfinite(p->T_m) || !std::isfinite(p->T_s) || !std::isfinite(p->T_l))
            return "phase-change temperatures must be finite";
        L->c_pl = p->c_pl;
        L->c_ref = 2.0 / (1.0 / p->c_pl + 1.0 / p->c_ps);  // Eq. B13
        L->sigma_s = p->sigma_s > 0.0 ? p->sigma_s : p->sigma;
        L->sigma_l = p->sigma_l > 0.0 ? p->sigma_l : p->sigma;
        L->T_s = p->T_l > p->T_s ? p->T_s : p->T_m;
        L->T_l = p->T_l > p->T_s ? p->T_l : p->T_m;
        L->L_a = p->c_pl * dT / p->St;  // St = c_pl dT / L_a
        L->alpha_l = L->alpha_f;
        L->alpha_s = L->alpha_f / p->alpha_ratio;
    }
    return nullptr;
}

}  // namespace

extern "C" {

lbm_status lbm_params_default(lbm_params* p) {
    if (!p) return LBM_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->nx = p->ny = p->nz = 1;
    p->storage = LBM_STORE_FP32;
    p->mapping = LBM_MAP_CAVITY;
    p->Ra = 1e3;
    p->Pr = 1.0;
    p->J = 1.0;
    p->sigma = 1.0;
    p->Gamma = 1.0;
    p->Ma = 0.1;
    p->dT = 1.0;
    p->T0 = 0.5;
    p->rho0 = 1.0;
    p->varpi = 0.5;
    p->s_e = p->s_eps = p->s_q = p->s_pi = 1.1;
    p->s_m = 1.2;
    p->zeta_T = 1.0;
    p->zeta_e = p->zeta_nu = 1.2;
    p->gravity_axis = 2;
    p->gravity_sign = -1;
    p->T_init = 0.5;
    p->T_m = 0.5;
    p->St = 1.0;
    p->c_pl = p->c_ps = 1.0;
    p->sigma_s = p->sigma_l = -1.0;
    p->alpha_ratio = 1.0;
    p->q_flow = 19;
    return LBM_OK;
}

lbm_status lbm_derive_lattice(const lbm_params* p, lbm_lattice* out) {
    if (!p || !out) return LBM_EINVAL;
    lbm_lattice L;
    if (derive(p, &L)) return LBM_EINVAL;
    *out = L;
    return LBM_OK;
}

const char* lbm_status_string(lbm_status s) {
    switch (s) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ENOMEM: return "out of device memory";
        case LBM_ECUDA: return "CUDA error";
        case LBM_EUNSTABLE: return "non-finite state";
        case LBM_ESTATE: return "call not allowed in the current state";
        case LBM_ETIMEOUT: return "a device-side wait timed out";
    }
    return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : "null context"; }

long long lbm_steps_done(const lbm_ctx* c) { return c ? c->steps : -1; }

}  // extern "C"

namespace {

// Per-launch parameter block from the lattice and the current medium.
void fill_kparams(lbm_ctx* c) {
    const lbm_params& p = c->prm;
    const lbm_lattice& L = c->lat;
    KParams& k = c->kp;
    k = KParams{};
    k.nx = p.nx;
    k.ny = p.ny;
    k.nz = p.nz;
    k.nyz = p.ny * p.nz;
    k.block_threads = c->block_threads;
    // all 26 planes of a copy and a site index within one plane addressed by an int offset
    k.off32 = (long long)(lbm::kQ + lbm::kQT + 1) * c->sq <= (long long)INT_MAX ? 1 : 0;
    k.enthalpy = L.enthalpy;
    k.flow_off = L.flow_off;
    if (L.enthalpy) {
        const double Es = L.sigma_s * L.c_pl * L.T_s;
        const double El = L.sigma_l * L.c_pl * L.T_l + L.phi * L.L_a;
        k.ent_Es = (float)Es;
        k.ent_El = (float)El;
        k.ent_is = (float)(1.0 / (L.sigma_s * L.c_pl));
        k.ent_il = (float)(1.0 / (L.sigma_l * L.c_pl));
        k.ent_Ts = (float)L.T_s;
        k.ent_Tl = (float)L.T_l;
        k.ent_idE = El > Es ? (float)(1.0 / (El - Es)) : 0.0f;
        k.c_pl = (float)L.c_pl;
        k.c_ref = (float)L.c_ref;
        k.alpha_s = (float)L.alpha_s;
        k.alpha_l = (float)L.alpha_l;
        k.inv_csT2 = (float)(3.0 / L.varpi);
    }
    k.storage = p.storage;
    k.om0 = (float)(1.0 - L.varpi);
    k.om1 = (float)(L.varpi / 6.0);
    k.iom0 = (float)(1.0 / (1.0 - L.varpi));
    k.iom1 = (float)(6.0 / L.varpi);
    k.ns = c->ns;
    k.sq = c->sq;
    for (int f = 0; f < 6; ++f) {
        unsigned bit = 1u << f;
        if (p.flow_bc[f] == LBM_FLOW_PERIODIC) k.per_mask |= bit;
        if (p.flow_bc[f] == LBM_FLOW_WALL) k.wall_mask |= bit;
        if (p.flow_bc[f] == LBM_FLOW_VELOCITY) k.vel_mask |= bit;
        if (p.flow_bc[f] == LBM_FLOW_NEE) k.nee_mask |= bit;
        k.face_dT[f] = (float)(p.face_T[f] - L.T0);
        k.heat_kind[f] = p.heat_bc[f];
        // anti-bounce-back term 2 omega_i sigma (T_w - T0) in deviation form, omega_i = varpi/6
        // enthalpy model: full values, weight varpi c_ref / 6 (Eq. B12)
        k.heat_abb[f] = L.enthalpy ? (float)(2.0 * (L.varpi / 6.0) * L.c_ref * p.face_T[f])
                                   : (float)(2.0 * (L.varpi / 6.0) * L.sigma * (p.face_T[f] - L.T0));
        for (int a = 0; a < 3; ++a) k.face_u[f][a] = (float)p.face_u[f][a];
    }
    double U = L.U_out > 0.0 ? L.U_out : 0.0;
    k.out_a = (float)(1.0 / (1.0 + U));
    k.out_b = (float)(U / (1.0 + U));
    // populations in units of 1 / fu (a power of two: every scaled constant is the FP32 one
    // times fu exactly)
    const double fu = p.storage == LBM_STORE_FP32 ? 1.0 : lbm::kFlowUnit;
    k.rho0 = (float)L.rho0;
    k.frho0 = (float)(fu * L.rho0);
    k.inv_fu = (float)(1.0 / fu);
    k.inv_rho0 = (float)(1.0 / (fu * L.rho0));
    k.sigma = (float)L.sigma;
    k.inv_sigma = (float)(1.0 / L.sigma);
    k.T0 = (float)L.T0;
    k.varpi = (float)L.varpi;
    k.s_e = (float)L.s[1];
    k.s_eps = (float)L.s[2];
    k.s_q = (float)L.s[4];
    k.s_nu = (float)L.s[9];
    k.s_pi = (float)L.s[10];
    k.s_m = (float)L.s[16];
    k.zeta_e = (float)L.zeta_e;
    k.zeta_nu = (float)L.zeta_nu;
    k.qf = L.q == 15 ? 15 : 19;
    {
        // per-moment collision factors: s_k / |M_k|^2 and (1 - s_k / 2) / |M_k|^2 (Eq. 9)
        auto a = [](double sk, double n2) { return (float)(sk / n2); };
        auto b = [](double sk, double n2) { return (float)((1.0 - 0.5 * sk) / n2); };
        double se = L.s[1], seps = L.s[2], sq = L.s[4], snu = L.s[9], spi = L.s[10], sm = L.s[16];
        double c23 = 2.0 / 3.0 * L.rho0;
        k.ae = a(se, 2394.0);
        k.be = b(se, 2394.0);
        k.aeps = a(seps, 252.0);
        k.beps = b(seps, 252.0);
        k.aq = a(sq, 40.0);
        k.aqc = (float)(fu * (sq / 40.0 * c23));
        k.bqc = (float)(fu * ((1.0 - 0.5 * sq) / 40.0 * c23));
        k.anu36 = a(snu, 36.0);
        k.bnu36 = b(snu, 36.0);
        k.api72 = a(spi, 72.0);
        k.hbpi72 = (float)(0.5 * (1.0 - 0.5 * spi) / 72.0);
        k.anu12 = a(snu, 12.0);
        k.bnu12 = b(snu, 12.0);
        k.api24 = a(spi, 24.0);
        k.hbpi24 = (float)(0.5 * (1.0 - 0.5 * spi) / 24.0);
        k.anu4 = a(snu, 4.0);
        k.bnu4 = b(snu, 4.0);
        k.am8 = a(sm, 8.0);
        k.rho0_10 = (float)(fu * (L.rho0 / 10.0));
        // D3Q15 (Eq. A1 row norms: e 18, eps 360, q 40, 3p_xx 12, p_ww 4, p_xy.. 8, m_xyz 8)
        const double c73 = 7.0 / 3.0 * L.rho0;  // q_eq = -7/3 rho0 u (Eq. 15)
        k.ae15 = a(se, 18.0);
        k.be15 = b(se, 18.0);
        k.aeps15 = a(seps, 360.0);
        k.beps15 = b(seps, 360.0);
        k.aqc15 = (float)(sq / 40.0 * c73);
        k.bqc15 = (float)((1.0 - 0.5 * sq) / 40.0 * c73);
        k.anu8 = a(snu, 8.0);
        k.bnu8 = b(snu, 8.0);
        k.ze6 = (float)(L.zeta_e / 6.0);
        k.zn6 = (float)(L.zeta_nu / 6.0);
    }
    k.zeta_alpha = (float)L.zeta_alpha;
    for (int a = 0; a < 3; ++a) {
        k.buoy[a] = (float)L.buoy[a];
        k.accel[a] = (float)L.accel[a];
    }
    // uniform medium (Eq. 4, Eq. 28; Ergun's Eq. 6 when F_phi < 0)
    double phi = L.phi, K = L.K;
    double Fp = L.F_phi < 0.0 ? 1.75 / std::sqrt(150.0 * phi * phi * phi) : L.F_phi;
    double c_darcy = std::isinf(K) ? 0.0 : phi * L.nu / K;
    double c_forch = std::isinf(K) ? 0.0 : phi * Fp / std::sqrt(K);
    k.phi = (float)phi;
    k.inv_phi = (float)(1.0 / phi);
    k.c_darcy = (float)c_darcy;
    k.c_forch = (float)c_forch;
    k.l0 = (float)(0.5 * (1.0 + 0.5 * c_darcy));
    k.l1 = (float)(0.5 * c_forch);
    // heterogeneous medium
    k.phi_field = L.has_phi_field ? c->phi_dev : nullptr;
    double pr = L.phi_ref;
    double kc_ref = pr * pr * pr / ((1.0 - pr) * (1.0 - pr));
    k.kinf = std::isinf(K) ? 1 : 0;
    k.cK = k.kinf ? 1.0f : (float)(K / kc_ref);
    k.nu = (float)L.nu;
    k.F_phi = (float)L.F_phi;
    k.hetero_alpha = L.alpha_m >= 0.0 ? 1 : 0;
    k.alpha_f = (float)L.alpha_f;
    k.alpha_m = (float)(L.alpha_m >= 0.0 ? L.alpha_m : 0.0);
    k.inv_sig_csT2 = (float)(1.0 / (L.sigma * L.varpi / 3.0));
    if (!L.has_phi_field && L.alpha_m >= 0.0) {
        double ae = phi * L.alpha_f + (1.0 - phi) * L.alpha_m;
        k.zeta_alpha = (float)(1.0 / (0.5 + ae / (L.sigma * L.varpi / 3.0)));
        k.hetero_alpha = 0;
    }
}

// Waits for the context's stream; a staged load of the TMA step kernel that ran out of time
// since the last check (the kernel's device flag) makes the context LBM_ETIMEOUT (sticky), so
// that no call returns results computed from a step that stopped early.
lbm_status sync_ctx(lbm_ctx* c) {
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    if (c->tma_err) {
        int flag = 0;
        LBM_CUDA(cudaMemcpy(&flag, c->tma_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            c->sticky = LBM_ETIMEOUT;
            return fail(c, LBM_ETIMEOUT, "a staged population load did not complete within 1 s");
        }
    }
    return LBM_OK;
}

lbm_status usable(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    if (c->sticky != LBM_OK) return c->sticky;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return LBM_OK;
}

float* cur_hist(lbm_ctx* c) { return c->hist[c->cur]; }

// Flow populations of the context's lattice (19 or 15) and whether logical plane q exists:
// f planes 0 .. Q-1, the D3Q7 planes at 19 .. 25 whatever the flow lattice.
int flow_q(const lbm_ctx* c) { return c->lat.q == 15 ? 15 : 19; }
bool has_plane(const lbm_ctx* c, int q) { return q < flow_q(c) || q >= lbm::kQ; }

// Start of logical population plane q of copy k (copies hold Q + 7 planes).
void* plane_ptr(const lbm_ctx* c, int k, int q) {
    if (c->aa) q = lbm::aa_swapped_plane(q);  // the state at rest is in the swapped layout
    const int phys = q < lbm::kQ ? q : flow_q(c) + (q - lbm::kQ);
    return static_cast<char*>(c->pop[k]) + (size_t)phys * (size_t)c->sq * c->elem;
}

// Element offset of a plane from the start of its copy (0 for a plane the lattice lacks).
int plane_off(const lbm_ctx* c, const void* base, const void* plane) {
    if (!plane) return 0;
    const long long off = (static_cast<const char*>(plane) - static_cast<const char*>(base)) /
                          (long long)c->elem;
    return off <= INT_MAX ? (int)off : 0;  // only used when KParams::off32 says all fit
}

// Plane tables of an AA context's single copy: `in_perm` / `out_perm` select the swapped
// layout (logical plane q at physical plane opp(q)) for the input / output side.
lbm::Planes aa_planes_at(const lbm_ctx* c, void* copy, bool in_perm, bool out_perm) {
    lbm::Planes pl;
    pl.base_in = copy;
    pl.base_out = copy;
    for (int q = 0; q < lbm::kQ + lbm::kQT; ++q) {
        const int pp = lbm::aa_swapped_plane(q);
        char* base = static_cast<char*>(copy);
        pl.in[q] = base + (size_t)(in_perm ? pp : q) * (size_t)c->sq * c->elem;
        pl.out[q] = base + (size_t)(out_perm ? pp : q) * (size_t)c->sq * c->elem;
        pl.off_in[q] = plane_off(c, pl.base_in, pl.in[q]);
        pl.off_out[q] = plane_off(c, pl.base_out, pl.out[q]);
    }
    pl.hin = nullptr;
    pl.hout = nullptr;
    pl.tin = nullptr;
    pl.tout = nullptr;
    return pl;
}

lbm::Planes aa_planes(const lbm_ctx* c, bool in_perm, bool out_perm) {
    return aa_planes_at(c, c->pop[0], in_perm, out_perm);
}

// Planes of a step that reads copy `from` and writes the other copy.
lbm::Planes planes(const lbm_ctx* c, int from) {
    lbm::Planes pl;
    const int to = from ^ 1;
    pl.base_in = c->pop[from];
    pl.base_out = c->pop[to];
    for (int q = 0; q < lbm::kQ + lbm::kQT; ++q) {
        pl.in[q] = has_plane(c, q) ? plane_ptr(c, from, q) : nullptr;
        pl.out[q] = has_plane(c, q) ? plane_ptr(c, to, q) : nullptr;
        pl.off_in[q] = plane_off(c, pl.base_in, pl.in[q]);
        pl.off_out[q] = plane_off(c, pl.base_out, pl.out[q]);
    }
    pl.hin = c->hist[from];
    pl.hout = c->hist[to];
    pl.tin = c->tplane[from];
    pl.tout = c->tplane[to];
    return pl;
}

lbm_status ensure_stage(lbm_ctx* c) {
    if (!c->stage) LBM_CUDA(cudaMalloc(&c->stage, sizeof(double) * 7 * (size_t)c->ns));
    return LBM_OK;
}

lbm_status ensure_mac(lbm_ctx* c) {
    if (!c->mac) LBM_CUDA(cudaMalloc(&c->mac, sizeof(float) * 9 * (size_t)c->ns));
    return LBM_OK;
}

// AA: the swapped layout every reader expects (a permutation after an odd number of steps).
lbm_status aa_settle(lbm_ctx* c) {
    if (!c->aa || c->aa_phase == 0) return LBM_OK;
    LBM_CUDA(lbm::launch_aa_normalize(c->kp, c->pl[0], c->stream));
    c->aa_phase = 0;
    return LBM_OK;
}

lbm_status reset_hist(lbm_ctx* c) {
    if (!c->outflow) return LBM_OK;
    LBM_CUDA(lbm::launch_hist_reset(c->kp, c->pl[c->cur], cur_hist(c), c->stream));
    return LBM_OK;
}

// Equilibrium state from device FP64 fields (or uniform values).
lbm_status init_state(lbm_ctx* c, const double* T_dev, const double* u_dev, double T_uniform) {
    // the equilibrium goes into the current copy: the planes that read copy `cur ^ 1` write it
    LBM_CUDA(lbm::launch_init_eq(c->kp, c->pl[c->cur ^ 1], T_dev, u_dev, T_uniform, c->stream));
    lbm_status s = reset_hist(c);
    if (s != LBM_OK) return s;
    c->steps = 0;
    c->have_prev = false;
    c->aa_phase = 0;
    return LBM_OK;
}

// cuTensorMapEncodeTiled, taken from the driver through the runtime (no link to libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor maps of both population copies for the TMA step kernel: the Q + 7 planes of a copy
// as (x, y, z, plane) with strides nx, nx ny and sq elements, and the FP32 temperature plane
// of the 16-bit formats as (x, y, z); boxes of 64 and 72 x 4 sites.  Out-of-range box
// elements are filled with zeros (the kernel never uses them).
lbm_status encode_tma_maps(lbm_ctx* c) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
        return fail(c, LBM_EINVAL, "cuTensorMapEncodeTiled is not available");
    const EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
    const lbm_params& p = c->prm;
    const cuuint64_t es = c->elem;
    const cuuint64_t nplanes = (cuuint64_t)(flow_q(c) + lbm::kQT);
    const cuuint64_t pdim[4] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz, nplanes};
    const cuuint64_t pstr[3] = {p.nx * es, (cuuint64_t)p.nx * p.ny * es, (cuuint64_t)c->sq * es};
    const cuuint64_t tdim[3] = {(cuuint64_t)p.nx, (cuuint64_t)p.ny, (cuuint64_t)p.nz};
    const cuuint64_t tstr[2] = {p.nx * 4ull, (cuuint64_t)p.nx * p.ny * 4ull};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt =
        es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    for (int k = 0; k < 2; ++k) {
        lbm::TmaMaps& m = c->tmaps[k];
        std::memset(&m, 0, sizeof(m));
        for (int wide = 0; wide < 2; ++wide) {
            const cuuint32_t bx = wide ? 72 : 64;
            const cuuint32_t pbox[4] = {bx, (cuuint32_t)lbm::kTmaTileY, 1, 1};
            CUresult r = encode(wide ? &m.pop72 : &m.pop64, dt, 4, c->pop[k], pdim, pstr, pbox,
                                ones, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(c, LBM_EINVAL, "cuTensorMapEncodeTiled(populations) failed: %d", (int)r);
            if (!c->tplane[k]) continue;
            r = encode(wide ? &m.t72 : &m.t64, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->tplane[k],
                       tdim, tstr, pbox, ones, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail(c, LBM_EINVAL, "cuTensorMapEncodeTiled(temperature) failed: %d", (int)r);
        }
    }
    return LBM_OK;
}

// The steady-state residual in two halves, so that a caller holding many contexts on one
// stream (the serving loop) synchronises once for all of them.  residual_launch queues the
// macroscopic fields of the current state, the reduction against the previous snapshot and
// the copy of its sums into the pinned mirror; residual_collect (after the stream has been
// synchronised) turns the sums into r_u, r_T and makes the new fields the snapshot.
lbm_status residual_launch(lbm_ctx* c) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if ((st = aa_settle(c)) != LBM_OK) return st;
    if ((st = ensure_mac(c)) != LBM_OK) return st;
    float* cu = c->mac + (size_t)(c->snap ^ 1) * 4 * c->ns;  // new fields
    float* cT = cu + 3 * c->ns;
    const float* pu = c->mac + (size_t)c->snap * 4 * c->ns;  // snapshot of the previous call
    const float* pT = pu + 3 * c->ns;
    LBM_CUDA(lbm::launch_macros(c->kp, c->outflow, c->pl[c->cur], nullptr, cu, cT, c->stream));
    if (!c->have_prev) {  // first call: no snapshot yet, compare the fields with themselves
        pu = cu;
        pT = cT;
    }
    const int nr = lbm::residual_blocks(c->ns);
    LBM_CUDA(lbm::launch_residual(cu, cT, pu, pT, c->ns, c->partials, nr, c->dres, c->stream));
    LBM_CUDA(cudaMemcpyAsync(c->hres, c->dres, sizeof(double) * 5, cudaMemcpyDeviceToHost,
                             c->stream));
    return LBM_OK;
}

lbm_status residual_collect(lbm_ctx* c, double* r_u, double* r_T) {
    const double* h = c->hres;
    const bool first = !c->have_prev;
    c->snap ^= 1;
    c->have_prev = true;
    if (h[4] > 0.0) return fail(c, LBM_EUNSTABLE, "velocity or temperature is not finite");
    // relative change; a field that is zero and unchanged has residual 0
    auto rel = [](double num, double den) {
        return den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? HUGE_VAL : 0.0);
    };
    double ru = first ? HUGE_VAL : rel(h[0], h[1]);
    double rT = first ? HUGE_VAL : rel(h[2], h[3]);
    if (r_u) *r_u = ru;
    if (r_T) *r_T = rT;
    return LBM_OK;
}

// Whether the paired step kernel can run a context.
bool pair_eligible(const lbm_ctx* c) {
    return flow_q(c) == 19 && !c->lat.enthalpy && !c->lat.node_walls && !c->aa &&
           c->prm.nx % 2 == 0 && c->kp.off32;
}

// A ping-pong context moved to the AA scheme (aa_eligible lattices): the AA layout at rest
// holds logical plane q at physical plane opp(q), so the current copy's planes are copied,
// permuted, into the other copy, which becomes the single copy; the current copy is freed.
// The populations are not changed, only where they are kept.
lbm_status convert_to_aa(lbm_ctx* c) {
    if (c->aa) return LBM_OK;
    if (!aa_eligible(&c->prm, c->lat))
        return fail(c, LBM_EINVAL, "this lattice cannot run the AA scheme");
    void* src = c->pop[c->cur];
    void* dst = c->pop[c->cur ^ 1];
    const size_t plane = (size_t)c->sq * c->elem;
    for (int q = 0; q < lbm::kQ + lbm::kQT; ++q)
        LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + (size_t)lbm::aa_swapped_plane(q) * plane,
                                 static_cast<const char*>(src) + (size_t)q * plane,
                                 (size_t)c->ns * c->elem, cudaMemcpyDeviceToDevice, c->stream));
    LBM_CUDA(cudaStreamSynchronize(c->stream));
    LBM_CUDA(cudaFree(src));
    c->pop[0] = dst;
    c->pop[1] = nullptr;
    c->cur = 0;
    c->aa = true;
    c->aa_phase = 0;
    c->lat.scheme = LBM_SCHEME_AA;
    if (c->step_kernel == LBM_KERNEL_PAIRED) c->step_kernel = LBM_KERNEL_PLAIN;
    c->pl[0] = aa_planes(c, true, false);
    c->pl[1] = aa_planes(c, false, true);
    c->pw = aa_planes(c, true, true);
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_create(const lbm_params* p, void* stream, lbm_ctx** out) {
    if (!p || !out) return LBM_EINVAL;
    lbm_lattice L;
    if (derive(p, &L)) return LBM_EINVAL;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ENOMEM;
    c->prm = *p;
    c->lat = L;
    c->ns = (long long)p->nx * p->ny * p->nz;
    c->sq = (c->ns + 63) / 64 * 64;  // 256-byte aligned population planes
    c->nyz = (long long)p->ny * p->nz;
    c->outflow = p->flow_bc[1] == LBM_FLOW_OUTFLOW;
    c->elem = p->storage == LBM_STORE_FP32 ? sizeof(float) : 2;
    lbm_status st = LBM_OK;
    // the device of a caller's stream, else the calling thread's current device
    cudaError_t e = stream ? cudaStreamGetDevice((cudaStream_t)stream, &c->device)
                           : cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaSetDevice(c->device);
    if (e != cudaSuccess) {
        st = cuda_fail(c, e, "selecting the device");
    } else if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) st = cuda_fail(c, e, "cudaStreamCreate");
        else c->own_stream = true;
    }
    // AUTO: ping-pong while both copies fit in the free device memory (auto_mem_limit, in
    // bytes, caps that figure), else AA where the lattice allows it
    if (st == LBM_OK && p->scheme == LBM_SCHEME_AUTO && aa_eligible(p, c->lat)) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "cudaMemGetInfo");
        } else {
            unsigned long long avail = fr;
            if (p->auto_mem_limit > 0 && p->auto_mem_limit < avail) avail = p->auto_mem_limit;
            if (footprint_of(p, c->lat, 0) > avail) c->lat.scheme = LBM_SCHEME_AA;
        }
    }
    c->aa = c->lat.scheme == LBM_SCHEME_AA;
    L = c->lat;
    size_t pop_bytes = c->elem * (size_t)((L.q == 15 ? 15 : lbm::kQ) + lbm::kQT) * (size_t)c->sq;
    for (int k = 0; k < (c->aa ? 1 : 2) && st == LBM_OK; ++k) {
        e = cudaMalloc(&c->pop[k], pop_bytes);
        if (e != cudaSuccess) st = cuda_fail(c, e, "cudaMalloc(populations)");
        if (st == LBM_OK && c->outflow) {
            e = cudaMalloc(&c->hist[k], sizeof(float) * lbm::kOutSlots * (size_t)c->nyz);
            if (e != cudaSuccess) st = cuda_fail(c, e, "cudaMalloc(outflow history)");
        }
        if (st == LBM_OK && p->storage != LBM_STORE_FP32) {
            e = cudaMalloc(&c->tplane[k], sizeof(float) * (size_t)c->ns);
            if (e != cudaSuccess) st = cuda_fail(c, e, "cudaMalloc(temperature plane)");
        }
    }
    if (st == LBM_OK) {
        int nr = lbm::reduction_blocks();
        size_t prof = (size_t)(p->nx > p->ny ? p->nx : p->ny);
        if ((e = cudaMalloc(&c->partials, sizeof(double) * 5 * nr)) != cudaSuccess ||
            (e = cudaMalloc(&c->profile, sizeof(double) * prof)) != cudaSuccess ||
            (e = cudaMalloc(&c->dres, sizeof(double) * 8)) != cudaSuccess ||
            (e = cudaMallocHost(&c->hres, sizeof(double) * 8)) != cudaSuccess)
            st = cuda_fail(c, e, "cudaMalloc(scratch)");
    }
    if (st == LBM_OK) {
        fill_kparams(c);
        // the paired kernel where it applies (bit-identical, faster in every measured case)
        if (pair_eligible(c)) c->step_kernel = LBM_KERNEL_PAIRED;
        if (c->aa) {
            c->pl[0] = aa_planes(c, true, false);
            c->pl[1] = aa_planes(c, false, true);
            c->pw = aa_planes(c, true, true);
        } else {
            c->pl[0] = planes(c, 0);
            c->pl[1] = planes(c, 1);
        }
        st = init_state(c, nullptr, nullptr, p->T_init);
    }
    if (st == LBM_OK) {
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) st = cuda_fail(c, e, "initialisation");
    }
    if (st != LBM_OK) {
        lbm_destroy(c);
        return st;
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->pop[k]);
        cudaFree(c->hist[k]);
        cudaFree(c->tplane[k]);
    }
    cudaFree(c->phi_dev);
    cudaFree(c->partials);
    cudaFree(c->profile);
    cudaFree(c->dres);
    cudaFreeHost(c->hres);
    cudaFree(c->stage);
    cudaFree(c->mac);
    cudaFree(c->tma_err);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

lbm_status lbm_set_medium(lbm_ctx* c, const float* phi_field, double phi, double K,
                          double F_phi, double alpha_m, double phi_ref) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    lbm_lattice L = c->lat;
    double mean = phi;
    if (phi_field && L.enthalpy)
        return fail(c, LBM_EINVAL, "the enthalpy model takes a uniform medium");
    if (phi_field) {
        double sum = 0.0;
        for (long long s = 0; s < c->ns; ++s) {
            double v = phi_field[s];
            if (!(v > 0.0 && v < 1.0)) return fail(c, LBM_EINVAL, "phi_field[%lld] = %g outside (0, 1)", s, v);
            sum += v;
        }
        mean = sum / (double)c->ns;
    } else if (!(phi > 0.0 && phi <= 1.0)) {
        return fail(c, LBM_EINVAL, "phi = %g outside (0, 1]", phi);
    }
    if (K <= 0.0) K = c->prm.Da > 0.0 ? c->prm.Da * L.L * L.L : HUGE_VAL;
    if (std::isnan(K)) return fail(c, LBM_EINVAL, "K is NaN");
    if (!std::isfinite(F_phi) && !(F_phi < 0.0)) return fail(c, LBM_EINVAL, "F_phi must be finite");
    if (phi_ref <= 0.0) phi_ref = mean;
    if (phi_field && !(phi_ref > 0.0 && phi_ref < 1.0))
        return fail(c, LBM_EINVAL, "phi_ref = %g outside (0, 1)", phi_ref);
    L.phi = phi_field ? mean : phi;
    L.K = K;
    L.F_phi = F_phi < 0.0 ? -1.0 : F_phi;
    L.alpha_m = alpha_m < 0.0 ? -1.0 : alpha_m;
    L.phi_ref = phi_ref;
    L.has_phi_field = phi_field ? 1 : 0;
    double csT2 = L.varpi / 3.0;
    double ae = alpha_m < 0.0 ? L.Gamma * L.alpha_f : L.phi * L.alpha_f + (1.0 - L.phi) * alpha_m;
    L.zeta_alpha = 1.0 / (0.5 + ae / (L.sigma * csT2));  // Eq. 41
    if (!rate_ok(L.zeta_alpha)) return fail(c, LBM_EINVAL, "zeta_alpha outside (0, 2)");
    if (phi_field) {
        if (!c->phi_dev) LBM_CUDA(cudaMalloc(&c->phi_dev, sizeof(float) * (size_t)c->ns));
        LBM_CUDA(cudaMemcpyAsync(c->phi_dev, phi_field, sizeof(float) * (size_t)c->ns,
                                 cudaMemcpyHostToDevice, c->stream));
    }
    if (lbm_status s_ = sync_ctx(c)) return s_;
    c->lat = L;
    fill_kparams(c);
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int nsteps) {
    NvtxRange range_("lbm_step");
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps < 0");
    if (c->aa) {
        for (int t = 0; t < nsteps; ++t) {
            const bool local = c->aa_phase == 1;
            LBM_CUDA(lbm::launch_aa_step(c->kp, local, c->pl[local ? 1 : 0], c->pw, c->pdl,
                                         c->stream));
            c->aa_phase ^= 1;
            c->steps++;
        }
        return LBM_OK;
    }
    for (int t = 0; t < nsteps; ++t) {
        int nxt = c->cur ^ 1;
        c->kp.reverse = c->cur;  // alternate sweep directions (sweep_block)
        if (c->step_kernel == LBM_KERNEL_PAIRED)
            LBM_CUDA(lbm::launch_step_pair(c->kp, c->outflow, c->pl[c->cur], c->pdl, c->stream));
        else if (c->step_kernel == LBM_KERNEL_TMA)
            LBM_CUDA(lbm::launch_step_tma(c->kp, c->outflow, c->pl[c->cur], c->tmaps[c->cur],
                                          c->tma_blocks, c->tma_extra_tx, c->tma_err, c->pdl,
                                          c->stream));
        else
            LBM_CUDA(lbm::launch_step(c->kp, c->outflow, c->pl[c->cur], c->pdl, c->stream));
        c->cur = nxt;
        c->steps++;
    }
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    return sync_ctx(c);
}

lbm_status lbm_init_equilibrium(lbm_ctx* c, const double* T_field, const double* u_field,
                                double T_uniform) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if (!std::isfinite(T_uniform)) return fail(c, LBM_EINVAL, "T_uniform must be finite");
    const double* Td = nullptr;
    const double* ud = nullptr;
    if (T_field || u_field) {
        if ((st = ensure_stage(c)) != LBM_OK) return st;
        if (T_field) {
            LBM_CUDA(cudaMemcpyAsync(c->stage, T_field, sizeof(double) * c->ns,
                                     cudaMemcpyHostToDevice, c->stream));
            Td = c->stage;
        }
        if (u_field) {
            LBM_CUDA(cudaMemcpyAsync(c->stage + c->ns, u_field, sizeof(double) * 3 * c->ns,
                                     cudaMemcpyHostToDevice, c->stream));
            ud = c->stage + c->ns;
        }
    }
    if ((st = init_state(c, Td, ud, T_uniform)) != LBM_OK) return st;
    if (lbm_status s_ = sync_ctx(c)) return s_;
    return LBM_OK;
}

// Weight that multiplies a stored value of plane q: 1 for FP32, w_i or omega_i for 16 bits.
static double plane_scale(const lbm_ctx* c, int q) {
    if (c->prm.storage == LBM_STORE_FP32) return 1.0;
    const lbm_lattice& L = c->lat;
    if (q < lbm::kQ) return 1.0 / lbm::kFlowUnit;  // D3Q19 only
    return q == lbm::kQ ? 1.0 - L.varpi : L.varpi / 6.0;
}

static double plane_offset(const lbm_ctx* c, int q) {
    // w_i rho0 for the flow planes (D3Q19 weights under Eq. 24, D3Q15 under Eq. 18),
    // omega_i sigma T0 for D3Q7 (Eq. 42)
    const lbm_lattice& L = c->lat;
    if (q < lbm::kQ) {
        double w = L.q == 15 ? (q == 0 ? 2.0 / 9.0 : (q <= 6 ? 1.0 / 9.0 : 1.0 / 72.0))
                             : (q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0));
        return w * L.rho0;
    }
    if (L.enthalpy) return 0.0;  // D3Q7 planes hold the full enthalpy populations
    int i = q - lbm::kQ;
    double om = i == 0 ? 1.0 - L.varpi : L.varpi / 6.0;
    return om * L.sigma * L.T0;
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* f, const double* g) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if (!f || !g) return fail(c, LBM_EINVAL, "f and g are required");
    if ((st = ensure_stage(c)) != LBM_OK) return st;
    const bool tshift = c->prm.storage != LBM_STORE_FP32;  // D3Q7 stored against local T
    const int nq = tshift ? lbm::kQ : lbm::kQ + lbm::kQT;
    for (int q = 0; q < nq; ++q) {
        if (!has_plane(c, q)) continue;
        const double* src = q < lbm::kQ ? f + (size_t)q * c->ns : g + (size_t)(q - lbm::kQ) * c->ns;
        double* stg = c->stage + (size_t)(q & 3) * c->ns;  // rotate 4 staging planes
        LBM_CUDA(cudaMemcpyAsync(stg, src, sizeof(double) * c->ns, cudaMemcpyHostToDevice,
                                 c->stream));
        LBM_CUDA(lbm::launch_plane_to_dev(c->prm.storage, stg, plane_ptr(c, c->cur, q),
                                          plane_offset(c, q), plane_scale(c, q), c->ns, c->stream));
    }
    if (tshift) {
        LBM_CUDA(cudaMemcpyAsync(c->stage, g, sizeof(double) * lbm::kQT * c->ns,
                                 cudaMemcpyHostToDevice, c->stream));
        LBM_CUDA(lbm::launch_g_to_dev(c->kp, c->pl[c->cur ^ 1], c->stage, c->stream));
    }
    if ((st = reset_hist(c)) != LBM_OK) return st;
    c->have_prev = false;
    c->aa_phase = 0;  // the whole state was written in the swapped layout
    if (lbm_status s_ = sync_ctx(c)) return s_;
    return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, double* f, double* g) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if ((st = aa_settle(c)) != LBM_OK) return st;
    if ((st = ensure_stage(c)) != LBM_OK) return st;
    const bool tshift = c->prm.storage != LBM_STORE_FP32;
    const int nq = tshift ? lbm::kQ : lbm::kQ + lbm::kQT;
    for (int q = 0; q < nq; ++q) {
        if (!has_plane(c, q)) continue;
        double* dst = q < lbm::kQ ? (f ? f + (size_t)q * c->ns : nullptr)
                                  : (g ? g + (size_t)(q - lbm::kQ) * c->ns : nullptr);
        if (!dst) continue;
        double* stg = c->stage + (size_t)(q & 3) * c->ns;
        LBM_CUDA(lbm::launch_plane_to_host(c->prm.storage, plane_ptr(c, c->cur, q), stg,
                                           plane_offset(c, q), plane_scale(c, q), c->ns, c->stream));
        LBM_CUDA(cudaMemcpyAsync(dst, stg, sizeof(double) * c->ns, cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    if (tshift && g) {
        // the FP64 planes must not be overwritten while an f copy above is in flight: the
        // stream orders the kernel after those copies
        LBM_CUDA(lbm::launch_g_to_host(c->kp, c->pl[c->cur], c->stage, c->stream));
        LBM_CUDA(cudaMemcpyAsync(g, c->stage, sizeof(double) * lbm::kQT * c->ns,
                                 cudaMemcpyDeviceToHost, c->stream));
    }
    if (lbm_status s_ = sync_ctx(c)) return s_;
    return LBM_OK;
}

// ---- raw state I/O -------------------------------------------------------------------------
namespace {
struct StateHeader {  // 128 bytes at the start of a state blob
    char magic[8];    // "LBMSTATE"
    int version;      // 2 (the 16-bit flow planes hold deviations in units of 1 / kFlowUnit)
    int nx, ny, nz;
    int q, storage, scheme;
    long long steps;
    unsigned long long pop_bytes, tplane_bytes, hist_bytes;
    char reserved[56];
};
static_assert(sizeof(StateHeader) == 128, "state header size");

StateHeader state_header(const lbm_ctx* c) {
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "LBMSTATE", 8);
    h.version = 2;
    h.nx = c->prm.nx;
    h.ny = c->prm.ny;
    h.nz = c->prm.nz;
    h.q = flow_q(c);
    h.storage = c->prm.storage;
    h.scheme = c->lat.scheme;
    h.steps = c->steps;
    h.pop_bytes = (unsigned long long)(flow_q(c) + lbm::kQT) * (unsigned long long)c->sq * c->elem;
    h.tplane_bytes = c->tplane[0] ? sizeof(float) * (unsigned long long)c->ns : 0ull;
    h.hist_bytes = c->outflow ? sizeof(float) * lbm::kOutSlots * (unsigned long long)c->nyz : 0ull;
    return h;
}
}  // namespace

lbm_status lbm_state_bytes(const lbm_ctx* c, unsigned long long* bytes) {
    if (!c || !bytes) return LBM_EINVAL;
    const StateHeader h = state_header(c);
    *bytes = sizeof(StateHeader) + h.pop_bytes + h.tplane_bytes + h.hist_bytes;
    return LBM_OK;
}

lbm_status lbm_save_state(lbm_ctx* c, void* host, unsigned long long bytes) {
    NvtxRange range_("lbm_save_state");
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    const StateHeader h = state_header(c);
    if (!host || bytes < sizeof(h) + h.pop_bytes + h.tplane_bytes + h.hist_bytes)
        return fail(c, LBM_EINVAL, "state buffer missing or smaller than lbm_state_bytes");
    if ((st = aa_settle(c)) != LBM_OK) return st;
    char* out = static_cast<char*>(host);
    std::memcpy(out, &h, sizeof(h));
    out += sizeof(h);
    LBM_CUDA(cudaMemcpyAsync(out, c->pop[c->cur], h.pop_bytes, cudaMemcpyDeviceToHost, c->stream));
    out += h.pop_bytes;
    if (h.tplane_bytes) {
        LBM_CUDA(cudaMemcpyAsync(out, c->tplane[c->cur], h.tplane_bytes, cudaMemcpyDeviceToHost,
                                 c->stream));
        out += h.tplane_bytes;
    }
    if (h.hist_bytes)
        LBM_CUDA(cudaMemcpyAsync(out, c->hist[c->cur], h.hist_bytes, cudaMemcpyDeviceToHost,
                                 c->stream));
    return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* host, unsigned long long bytes) {
    NvtxRange range_("lbm_load_state");
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    const StateHeader mine = state_header(c);
    StateHeader h;
    if (!host || bytes < sizeof(h)) return fail(c, LBM_EINVAL, "state buffer missing");
    std::memcpy(&h, host, sizeof(h));
    if (std::memcmp(h.magic, mine.magic, 8) != 0 || h.version != mine.version)
        return fail(c, LBM_EINVAL, "not a state blob of this library version");
    if (h.nx != mine.nx || h.ny != mine.ny || h.nz != mine.nz || h.q != mine.q ||
        h.storage != mine.storage || h.scheme != mine.scheme || h.pop_bytes != mine.pop_bytes ||
        h.tplane_bytes != mine.tplane_bytes || h.hist_bytes != mine.hist_bytes)
        return fail(c, LBM_EINVAL, "state blob of a different lattice, format or scheme");
    if (bytes < sizeof(h) + h.pop_bytes + h.tplane_bytes + h.hist_bytes)
        return fail(c, LBM_EINVAL, "state buffer shorter than its header says");
    const char* in = static_cast<const char*>(host) + sizeof(h);
    LBM_CUDA(cudaMemcpyAsync(c->pop[c->cur], in, h.pop_bytes, cudaMemcpyHostToDevice, c->stream));
    in += h.pop_bytes;
    if (h.tplane_bytes) {
        LBM_CUDA(cudaMemcpyAsync(c->tplane[c->cur], in, h.tplane_bytes, cudaMemcpyHostToDevice,
                                 c->stream));
        in += h.tplane_bytes;
    }
    if (h.hist_bytes)
        LBM_CUDA(cudaMemcpyAsync(c->hist[c->cur], in, h.hist_bytes, cudaMemcpyHostToDevice,
                                 c->stream));
    c->steps = h.steps;
    c->have_prev = false;
    c->aa_phase = 0;
    return LBM_OK;
}

lbm_status lbm_macros_device(lbm_ctx* c, float* rho, float* u, float* T) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if ((st = aa_settle(c)) != LBM_OK) return st;
    LBM_CUDA(lbm::launch_macros(c->kp, c->outflow, c->pl[c->cur], rho, u, T, c->stream));
    return LBM_OK;
}

lbm_status lbm_macros(lbm_ctx* c, float* rho, float* u, float* T) {
    NvtxRange range_("lbm_macros");
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if ((st = aa_settle(c)) != LBM_OK) return st;
    if ((st = ensure_mac(c)) != LBM_OK) return st;
    float* half = c->mac + (size_t)(c->snap ^ 1) * 4 * c->ns;  // the half not holding the snapshot
    float* du = half;
    float* dT = half + 3 * c->ns;
    float* drho = c->mac + 8 * c->ns;
    LBM_CUDA(lbm::launch_macros(c->kp, c->outflow, c->pl[c->cur], rho ? drho : nullptr,
                                u ? du : nullptr, T ? dT : nullptr, c->stream));
    if (rho)
        LBM_CUDA(cudaMemcpyAsync(rho, drho, sizeof(float) * c->ns, cudaMemcpyDeviceToHost, c->stream));
    if (u)
        LBM_CUDA(cudaMemcpyAsync(u, du, sizeof(float) * 3 * c->ns, cudaMemcpyDeviceToHost, c->stream));
    if (T)
        LBM_CUDA(cudaMemcpyAsync(T, dT, sizeof(float) * c->ns, cudaMemcpyDeviceToHost, c->stream));
    if (lbm_status s_ = sync_ctx(c)) return s_;
    return LBM_OK;
}

lbm_status lbm_nusselt(lbm_ctx* c, int face, double* nu_avg, double* nu_profile, double* nu_mp) {
    NvtxRange range_("lbm_nusselt");
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if ((st = aa_settle(c)) != LBM_OK) return st;
    if (face < 0 || face > 5) return fail(c, LBM_EINVAL, "face must be 0..5");
    const bool node_wall = c->prm.heat_bc[face] == LBM_HEAT_NEE_DIRICHLET;
    if (c->prm.heat_bc[face] != LBM_HEAT_DIRICHLET && !node_wall)
        return fail(c, LBM_EINVAL, "face %d is not a Dirichlet (fixed temperature) face", face);
    int axis = face >> 1;
    int n[3] = {c->prm.nx, c->prm.ny, c->prm.nz};
    if (n[axis] < (node_wall ? 3 : 2))
        return fail(c, LBM_EINVAL, "Nusselt needs more sites normal to the face");
    int n1 = axis == 0 ? c->prm.ny : c->prm.nx;
    double scale = c->lat.L / c->lat.dT;
    LBM_CUDA(lbm::launch_nusselt(c->kp, c->outflow, c->pl[c->cur], face, c->prm.face_T[face],
                                 scale, c->profile, c->dres, c->stream));
    LBM_CUDA(cudaMemcpyAsync(c->hres, c->dres, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                             c->stream));
    if (nu_profile)
        LBM_CUDA(cudaMemcpyAsync(nu_profile, c->profile, sizeof(double) * n1,
                                 cudaMemcpyDeviceToHost, c->stream));
    if (lbm_status s_ = sync_ctx(c)) return s_;
    if (!std::isfinite(c->hres[0])) return fail(c, LBM_EUNSTABLE, "Nusselt number is not finite");
    if (nu_avg) *nu_avg = c->hres[0];
    if (nu_mp) *nu_mp = c->hres[1];
    return LBM_OK;
}

lbm_status lbm_sums(lbm_ctx* c, double* mass_dev, double* heat_dev) {
    NvtxRange range_("lbm_sums");
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if ((st = aa_settle(c)) != LBM_OK) return st;
    int nr = lbm::reduction_blocks();
    LBM_CUDA(lbm::launch_sums(c->kp, c->pl[c->cur], c->partials, nr, c->dres, c->stream));
    LBM_CUDA(cudaMemcpyAsync(c->hres, c->dres, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                             c->stream));
    if (lbm_status s_ = sync_ctx(c)) return s_;
    if (mass_dev) *mass_dev = c->hres[0];
    if (heat_dev) *heat_dev = c->hres[1];
    if (!std::isfinite(c->hres[0]) || !std::isfinite(c->hres[1]))
        return fail(c, LBM_EUNSTABLE, "population totals are not finite");
    return LBM_OK;
}

lbm_status lbm_residual(lbm_ctx* c, double* r_u, double* r_T) {
    NvtxRange range_("lbm_residual");
    lbm_status st = residual_launch(c);
    if (st != LBM_OK) return st;
    if ((st = sync_ctx(c)) != LBM_OK) return st;
    return residual_collect(c, r_u, r_T);
}

lbm_status lbm_set_step_kernel(lbm_ctx* c, int kernel) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if (kernel == LBM_KERNEL_PLAIN) {
        c->step_kernel = kernel;
        return LBM_OK;
    }
    if (kernel == LBM_KERNEL_PAIRED) {
        if (!pair_eligible(c))
            return fail(c, LBM_EINVAL, "the paired step kernel takes D3Q19 ping-pong lattices "
                                       "without node walls or enthalpy, with an even nx and "
                                       "fewer than ~82 M sites");
        c->step_kernel = kernel;
        return LBM_OK;
    }
    if (kernel != LBM_KERNEL_TMA) return fail(c, LBM_EINVAL, "unknown step kernel %d", kernel);
    const lbm_params& p = c->prm;
    if (flow_q(c) != 19 || c->lat.enthalpy || c->lat.node_walls)
        return fail(c, LBM_EINVAL, "the TMA step kernel takes D3Q19 without node walls or enthalpy");
    if (c->aa) return fail(c, LBM_EINVAL, "the TMA step kernel runs the ping-pong scheme");
    if (p.nx % lbm::kTmaTileX != 0 || p.ny < lbm::kTmaTileY)
        return fail(c, LBM_EINVAL, "the TMA step kernel needs nx %% %d == 0 and ny >= %d",
                    lbm::kTmaTileX, lbm::kTmaTileY);
    if ((st = encode_tma_maps(c)) != LBM_OK) return st;
    int blocks = 0, smem = 0;
    LBM_CUDA(lbm::tma_prepare(c->kp, c->outflow, &blocks, &smem));
    if (blocks <= 0) return fail(c, LBM_EINVAL, "the TMA step kernel does not fit on an SM");
    if (!c->tma_err) {
        LBM_CUDA(cudaMalloc(&c->tma_err, sizeof(int)));
        LBM_CUDA(cudaMemsetAsync(c->tma_err, 0, sizeof(int), c->stream));
        if (lbm_status s_ = sync_ctx(c)) return s_;
    }
    c->tma_blocks = blocks;
    c->step_kernel = kernel;
    return LBM_OK;
}

int lbm_get_step_kernel(const lbm_ctx* c) { return c ? c->step_kernel : -1; }

lbm_status lbm_bounds_report(long long* first_bad) {
    if (!first_bad) return LBM_EINVAL;
    int checked = 0;
    if (lbm::bounds_report(first_bad, &checked) != cudaSuccess) return LBM_ECUDA;
    return checked ? LBM_OK : LBM_EINVAL;
}

lbm_status lbm_set_launch(lbm_ctx* c, int block_threads, int dependent_launch) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if (block_threads != 0 && block_threads != 32 && block_threads != 64 && block_threads != 128 &&
        block_threads != 256)
        return fail(c, LBM_EINVAL, "block_threads must be 0, 32, 64, 128 or 256");
    if (dependent_launch < -1 || dependent_launch > 1)
        return fail(c, LBM_EINVAL, "dependent_launch must be -1, 0 or 1");
    if (block_threads) c->block_threads = block_threads;
    if (dependent_launch >= 0) c->pdl = dependent_launch != 0;
    fill_kparams(c);  // the block size travels in the kernel parameters
    return LBM_OK;
}

lbm_status lbm_test_tma_extra_wait(lbm_ctx* c, int bytes) {
    lbm_status st = usable(c);
    if (st != LBM_OK) return st;
    if (bytes < 0 || bytes > 4096) return fail(c, LBM_EINVAL, "bytes must be 0 .. 4096");
    c->tma_extra_tx = bytes;
    return LBM_OK;
}

lbm_status lbm_get_lattice(const lbm_ctx* c, lbm_lattice* out) {
    if (!c || !out) return LBM_EINVAL;
    *out = c->lat;
    return LBM_OK;
}

}  // extern "C"

// ---- batched launches --------------------------------------------------------------------------
#include <map>
#include <vector>

struct lbm_batch {
    std::vector<lbm_ctx*> ctx;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int block_threads = 64;
    int rows = 1;  // z-planes per block of the batched step
    struct Group {
        int storage = 0;
        bool het = false, outflow = false, enthalpy = false;
        bool aa = false;  // AA-scheme lattices (one copy each, stepped by batch_aa_kernel)
        bool off32 = false;  // the members' planes are addressed by 32-bit offsets
        bool pair = false;   // two x-adjacent sites per thread (batch_pair_kernel)
        int qf = 19;         // flow lattice: D3Q19 or D3Q15
        bool nee = false;    // node walls (non-equilibrium extrapolation)
        // each member stepped by its own single-lattice kernel (launched directly, not from
        // the graph), chosen by the tuner where that is faster than the fused launch
        bool solo = false;
        std::vector<int> members;           // indices into ctx
        lbm::BatchLattice* dtab = nullptr;  // device table
        // host mirror in pageable memory: an asynchronous copy from it stages the data before
        // returning, so the next call may refill it at once
        std::vector<lbm::BatchLattice> htab;
        int nblocks = 0;
        unsigned short* dblk = nullptr;     // block -> lattice map (device)
        size_t dblk_cap = 0;
        int dblk_threads = 0, dblk_rows = 0;  // layout the map was built for
        std::vector<unsigned short> hblk;
    };
    std::vector<Group> groups;
    std::map<int, cudaGraphExec_t> graphs;  // captured n-step sequences
    cudaEvent_t ev = nullptr;
    bool tuned = false;
    double last_pp_ms = 0.0, last_aa_ms = 0.0;  // the tuner's last scheme trial (per step)
    char err[256] = {0};
};

namespace {

lbm_status batch_fail(lbm_batch* b, lbm_status s, const char* what, cudaError_t e = cudaSuccess) {
    if (b) snprintf(b->err, sizeof(b->err), "%s%s%s", what, e != cudaSuccess ? ": " : "",
                    e != cudaSuccess ? cudaGetErrorString(e) : "");
    return s;
}

#define LBM_BCUDA(call)                                                     \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return batch_fail(b, LBM_ECUDA, #call, e_);  \
    } while (0)

void batch_clear_graphs(lbm_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Block layout of one lattice of a batch (x-extent, blocks along x and y; pair: nx / 2 pairs
// per row); returns its number of blocks.
int batch_layout(const lbm_ctx* c, bool pair, int block_threads, int rows, lbm::BatchLattice* L) {
    const int nx = pair ? c->prm.nx / 2 : c->prm.nx;
    L->bx = lbm::block_x(nx, block_threads);
    const int by = block_threads / L->bx;
    L->gx = (nx + L->bx - 1) / L->bx;
    L->gy = (c->prm.ny + by - 1) / by;
    return L->gx * L->gy * ((c->prm.nz + rows - 1) / rows);
}

// Host tables of every group from the contexts' current state and the block size.
void batch_fill_tables(lbm_batch* b) {
    for (auto& g : b->groups) {
        int off = 0;
        for (size_t k = 0; k < g.members.size(); ++k) {
            lbm_ctx* c = b->ctx[g.members[k]];
            lbm::BatchLattice& L = g.htab[k];
            L.p = c->kp;
            L.pl[0] = c->pl[0];
            L.pl[1] = c->pl[1];
            L.cur = c->aa ? c->aa_phase : c->cur;  // AA: 0 pull step next, 1 local step next
            L.block_begin = off;
            off += batch_layout(c, g.pair, b->block_threads, b->rows, &L);
        }
        g.nblocks = off;
    }
}

// The block -> lattice map of a table whose block_begin fields are set (nblocks blocks).
std::vector<unsigned short> batch_block_map(const std::vector<lbm::BatchLattice>& tab, int nblocks) {
    std::vector<unsigned short> blk((size_t)nblocks, 0);
    for (size_t k = 0; k < tab.size(); ++k) {
        const int end = k + 1 < tab.size() ? tab[k + 1].block_begin : nblocks;
        for (int i = tab[k].block_begin; i < end; ++i) blk[(size_t)i] = (unsigned short)k;
    }
    return blk;
}

// Order the batch stream after every context's pending work (and the reverse at the end).
lbm_status batch_join(lbm_batch* b, bool into_batch) {
    for (lbm_ctx* c : b->ctx) {
        if (c->stream == b->stream) continue;
        cudaStream_t from = into_batch ? c->stream : b->stream;
        cudaStream_t to = into_batch ? b->stream : c->stream;
        LBM_BCUDA(cudaEventRecord(b->ev, from));
        LBM_BCUDA(cudaStreamWaitEvent(to, b->ev, 0));
    }
    return LBM_OK;
}

// The steps of a group whose members run their own single-lattice kernels: all nsteps of one
// member, then the next (the members are independent; consecutive steps of one lattice find
// much of its state still in L2), step t of a member reading its copy cur ^ (t & 1) (tuning:
// always cur, so that only the other copy is written).
lbm_status batch_launch_solo(lbm_batch* b, lbm_batch::Group& g, int nsteps, bool tuning) {
    for (int k : g.members) {
        lbm_ctx* c = b->ctx[k];
        lbm::KParams kp = c->kp;
        for (int t = 0; t < nsteps; ++t) {
            const int from = c->cur ^ (tuning ? 0 : (t & 1));
            kp.reverse = from;  // alternate sweep directions, as lbm_step
            const lbm::Planes& pl = c->pl[from];
            LBM_BCUDA(g.pair ? lbm::launch_step_pair(kp, c->outflow, pl, c->pdl, b->stream)
                             : lbm::launch_step(kp, c->outflow, pl, c->pdl, b->stream));
        }
    }
    return LBM_OK;
}

// The fused launches of nsteps steps (the solo groups are left to batch_launch_solo).
// tuning: launches that leave the state unchanged, so AA groups (updated in place) are left out
lbm_status batch_launch_steps(lbm_batch* b, int nsteps, bool tuning) {
    for (int t = 0; t < nsteps; ++t)
        for (auto& g : b->groups) {
            if (g.solo) continue;
            if (g.aa) {
                if (!tuning)
                    LBM_BCUDA(lbm::launch_batch_aa(g.dtab, g.dblk, g.nblocks, b->block_threads,
                                                   b->rows, g.het, t & 1, b->stream));
                continue;
            }
            LBM_BCUDA(lbm::launch_batch_step(g.dtab, g.dblk, g.nblocks, b->block_threads, b->rows,
                                             g.storage, g.het, g.outflow, g.enthalpy, g.off32,
                                             g.pair, g.qf, g.nee, tuning ? 0 : (t & 1),
                                             b->stream));
        }
    return LBM_OK;
}

// Upload the lattice tables, and the block -> lattice map when the layout changed.
lbm_status batch_upload(lbm_batch* b) {
    batch_fill_tables(b);
    for (auto& g : b->groups) {
        LBM_BCUDA(cudaMemcpyAsync(g.dtab, g.htab.data(),
                                  sizeof(lbm::BatchLattice) * g.members.size(),
                                  cudaMemcpyHostToDevice, b->stream));
        if (g.dblk_threads == b->block_threads && g.dblk_rows == b->rows && g.dblk) continue;
        g.hblk = batch_block_map(g.htab, g.nblocks);
        if ((size_t)g.nblocks > g.dblk_cap) {
            // the map is sized once per layout; kernels of earlier launches may still read
            // the old one, so wait for them before freeing it
            LBM_BCUDA(cudaStreamSynchronize(b->stream));
            cudaFree(g.dblk);
            g.dblk = nullptr;
            LBM_BCUDA(cudaMalloc(&g.dblk, sizeof(unsigned short) * (size_t)g.nblocks));
            g.dblk_cap = (size_t)g.nblocks;
        }
        LBM_BCUDA(cudaMemcpyAsync(g.dblk, g.hblk.data(), sizeof(unsigned short) * g.hblk.size(),
                                  cudaMemcpyHostToDevice, b->stream));
        g.dblk_threads = b->block_threads;
        g.dblk_rows = b->rows;
    }
    return LBM_OK;
}

// Whether a ping-pong group could run the AA scheme (every member is eligible).
bool group_aa_eligible(const lbm_batch* b, const lbm_batch::Group& g) {
    if (g.aa) return false;
    for (int k : g.members)
        if (!aa_eligible(&b->ctx[k]->prm, b->ctx[k]->lat)) return false;
    return true;
}

// Milliseconds per step of one group at the batch's block shape: the ping-pong kernel in its
// state-preserving form (flip 0 writes only the non-current copies), or, with `aa`, the AA
// kernel run on scratch: each member's non-current copy, filled with its current state, is
// stepped in place as an AA copy, so the state stays untouched.
lbm_status time_group(lbm_batch* b, lbm_batch::Group& g, bool aa, float* ms_per_step) {
    const int nwarm = 2, ntime = 6;
    lbm::BatchLattice* dtab = g.dtab;
    unsigned short* dblk = g.dblk;
    int nblocks = g.nblocks;
    std::vector<lbm::BatchLattice> tab;
    std::vector<unsigned short> blk;
    if (aa) {
        tab = g.htab;
        for (size_t k = 0; k < g.members.size(); ++k) {
            lbm_ctx* c = b->ctx[g.members[k]];
            void* scratch = c->pop[c->cur ^ 1];
            LBM_BCUDA(cudaMemcpyAsync(scratch, c->pop[c->cur],
                                      (size_t)(lbm::kQ + lbm::kQT) * c->sq * c->elem,
                                      cudaMemcpyDeviceToDevice, b->stream));
            tab[k].pl[0] = aa_planes_at(c, scratch, true, false);
            tab[k].pl[1] = aa_planes_at(c, scratch, false, true);
            tab[k].cur = 0;
        }
        if (g.pair) {  // the AA kernel takes one site per thread: a layout of its own
            int off = 0;
            for (size_t k = 0; k < g.members.size(); ++k) {
                tab[k].block_begin = off;
                off += batch_layout(b->ctx[g.members[k]], false, b->block_threads, b->rows, &tab[k]);
            }
            nblocks = off;
            blk = batch_block_map(tab, nblocks);
            LBM_BCUDA(cudaMalloc(&dblk, sizeof(unsigned short) * blk.size()));
            LBM_BCUDA(cudaMemcpyAsync(dblk, blk.data(), sizeof(unsigned short) * blk.size(),
                                      cudaMemcpyHostToDevice, b->stream));
        }
        LBM_BCUDA(cudaMalloc(&dtab, sizeof(lbm::BatchLattice) * tab.size()));
        LBM_BCUDA(cudaMemcpyAsync(dtab, tab.data(), sizeof(lbm::BatchLattice) * tab.size(),
                                  cudaMemcpyHostToDevice, b->stream));
    }
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    for (int t = 0; t < nwarm + ntime && e == cudaSuccess; ++t) {
        if (t == nwarm) e = cudaEventRecord(t0, b->stream);
        if (e != cudaSuccess) break;
        e = aa ? lbm::launch_batch_aa(dtab, dblk, nblocks, b->block_threads, b->rows, g.het,
                                      t & 1, b->stream)
               : lbm::launch_batch_step(dtab, dblk, nblocks, b->block_threads, b->rows,
                                        g.storage, g.het, g.outflow, g.enthalpy, g.off32, g.pair,
                                        g.qf, g.nee, 0, b->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (aa) cudaFree(dtab);
    if (dblk != g.dblk) cudaFree(dblk);
    if (e != cudaSuccess) return batch_fail(b, LBM_ECUDA, "timing a group", e);
    *ms_per_step = ms / ntime;
    return LBM_OK;
}

// Milliseconds per step of a group's members stepped by their own kernels (tuning launches:
// the state is unchanged).
lbm_status time_solo(lbm_batch* b, lbm_batch::Group& g, float* ms_per_step) {
    const int nwarm = 2, ntime = 6;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    lbm_status st = LBM_OK;
    if (e == cudaSuccess) st = batch_launch_solo(b, g, nwarm, true);
    if (e == cudaSuccess && st == LBM_OK) e = cudaEventRecord(t0, b->stream);
    if (e == cudaSuccess && st == LBM_OK) st = batch_launch_solo(b, g, ntime, true);
    if (e == cudaSuccess && st == LBM_OK) e = cudaEventRecord(t1, b->stream);
    if (e == cudaSuccess && st == LBM_OK) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess && st == LBM_OK) e = cudaEventElapsedTime(&ms, t0, t1);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st != LBM_OK) return st;
    if (e != cudaSuccess) return batch_fail(b, LBM_ECUDA, "timing a group", e);
    *ms_per_step = ms / ntime;
    return LBM_OK;
}

// (Re)build the batch's kernel-variant groups and their device tables.
lbm_status batch_group(lbm_batch* b) {
    // group the lattices by kernel variant
    lbm_status st = LBM_OK;
    const int n = (int)b->ctx.size();
    for (auto& g : b->groups) {
        cudaFree(g.dtab);
        cudaFree(g.dblk);
    }
    b->groups.clear();
    for (int k = 0; k < n; ++k) {
        lbm_ctx* c = b->ctx[k];
        const int stg = c->prm.storage;
        const bool het = c->lat.has_phi_field != 0, outf = c->outflow;
        const bool ent = c->lat.enthalpy != 0, aa = c->aa, o32 = c->kp.off32 != 0;
        const bool pr = pair_eligible(c);  // two sites per thread where the paired kernel applies
        const int qf = flow_q(c);
        const bool nee = c->lat.node_walls != 0;
        lbm_batch::Group* grp = nullptr;
        for (auto& gr : b->groups)
            if (gr.storage == stg && gr.het == het && gr.outflow == outf && gr.enthalpy == ent &&
                gr.aa == aa && gr.off32 == o32 && gr.pair == pr && gr.qf == qf && gr.nee == nee)
                grp = &gr;
        if (!grp) {
            b->groups.emplace_back();
            grp = &b->groups.back();
            grp->storage = stg;
            grp->het = het;
            grp->outflow = outf;
            grp->enthalpy = ent;
            grp->aa = aa;
            grp->off32 = o32;
            grp->pair = pr;
            grp->qf = qf;
            grp->nee = nee;
        }
        grp->members.push_back(k);
    }
    for (auto& g : b->groups) {
        if (st != LBM_OK) break;
        size_t bytes = sizeof(lbm::BatchLattice) * g.members.size();
        g.htab.resize(g.members.size());
        if (cudaMalloc(&g.dtab, bytes) != cudaSuccess) st = LBM_ENOMEM;
    }
    return st;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, void* stream, lbm_batch** out) {
    if (!ctxs || n < 1 || !out) return LBM_EINVAL;
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ENOMEM;
    if (n > 65535) {  // the block -> lattice map holds 16-bit indices
        delete b;
        return LBM_EINVAL;
    }
    for (int k = 0; k < n; ++k) {
        lbm_ctx* c = ctxs[k];
        if (!c || c->sticky != LBM_OK) {
            delete b;
            return LBM_EINVAL;
        }
        for (lbm_ctx* o : b->ctx)
            if (o == c) {  // a lattice may appear once
                delete b;
                return LBM_EINVAL;
            }
        if (!b->ctx.empty() && c->device != b->ctx[0]->device) {
            delete b;
            return LBM_EINVAL;
        }
        b->ctx.push_back(c);
    }
    b->device = b->ctx[0]->device;
    lbm_status st = LBM_OK;
    cudaError_t e = cudaSetDevice(b->device);
    if (e == cudaSuccess) {
        if (stream) {
            b->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
            b->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) st = LBM_ECUDA;
    if (st == LBM_OK) st = batch_group(b);
    if (st != LBM_OK) {
        lbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_clear_graphs(b);
    for (auto& g : b->groups) {
        cudaFree(g.dtab);
        cudaFree(g.dblk);
    }
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

lbm_status lbm_batch_step(lbm_batch* b, int nsteps) {
    NvtxRange range_("lbm_batch_step");
    if (!b || nsteps < 0) return LBM_EINVAL;
    for (lbm_ctx* c : b->ctx)
        if (c->sticky != LBM_OK) return c->sticky;
    if (nsteps == 0) return LBM_OK;
    LBM_BCUDA(cudaSetDevice(b->device));
    lbm_status st = batch_join(b, true);
    if (st != LBM_OK) return st;
    if ((st = batch_upload(b)) != LBM_OK) return st;
    bool fused = false;
    for (auto& g : b->groups) fused = fused || !g.solo;
    auto it = b->graphs.find(nsteps);
    if (fused && it == b->graphs.end()) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        LBM_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        lbm_status ls = batch_launch_steps(b, nsteps, false);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (ls != LBM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return ls;
        }
        if (e != cudaSuccess) return batch_fail(b, LBM_ECUDA, "cudaStreamEndCapture", e);
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return batch_fail(b, LBM_ECUDA, "cudaGraphInstantiate", e);
        it = b->graphs.emplace(nsteps, exec).first;
    }
    if (fused) LBM_BCUDA(cudaGraphLaunch(it->second, b->stream));
    for (auto& g : b->groups)
        if (g.solo && (st = batch_launch_solo(b, g, nsteps, false)) != LBM_OK) return st;
    for (lbm_ctx* c : b->ctx) {
        if (c->aa) c->aa_phase ^= (nsteps & 1);
        else c->cur ^= (nsteps & 1);
        c->steps += nsteps;
    }
    return batch_join(b, false);
}

// Stage (1) of lbm_batch_tune: the block shape, timed without changing the lattices' state.
static lbm_status batch_tune_shape(lbm_batch* b, int* block_threads, int* rows) {
    bool timed = false;  // only ping-pong groups can be timed without changing the state
    for (auto& g : b->groups) timed = timed || !g.aa;
    if (!timed) {
        // a batch of AA lattices only: the shape measured fastest for the 64 seeded cavities
        // (GB300: 32 threads x 4 planes, 23.1k MLUPS against 20.3k at 64 x 1)
        if (b->block_threads != 32 || b->rows != 4) batch_clear_graphs(b);
        b->block_threads = 32;
        b->rows = 4;
        b->tuned = true;
        if (block_threads) *block_threads = b->block_threads;
        if (rows) *rows = b->rows;
        return LBM_OK;
    }
    LBM_BCUDA(cudaSetDevice(b->device));
    lbm_status st = batch_join(b, true);
    if (st != LBM_OK) return st;
    cudaEvent_t t0, t1;
    LBM_BCUDA(cudaEventCreate(&t0));
    LBM_BCUDA(cudaEventCreate(&t1));
    const int cand_t[4] = {32, 64, 128, 256};
    const int cand_r[3] = {1, 2, 4};
    int best = b->block_threads, best_rows = b->rows;
    float best_ms = 1e30f;
    for (int k = 0; k < 12 && st == LBM_OK; ++k) {
        b->block_threads = cand_t[k / 3];
        b->rows = cand_r[k % 3];
        // launches with flip 0 write only the non-current copy: the state is not changed
        if ((st = batch_upload(b)) != LBM_OK) break;
        if ((st = batch_launch_steps(b, 2, true)) != LBM_OK) break;  // warm-up
        cudaEventRecord(t0, b->stream);
        if ((st = batch_launch_steps(b, 5, true)) != LBM_OK) break;
        cudaEventRecord(t1, b->stream);
        cudaError_t e = cudaEventSynchronize(t1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) st = batch_fail(b, LBM_ECUDA, "tuning", e);
        else if (ms < best_ms) {
            best_ms = ms;
            best = b->block_threads;
            best_rows = b->rows;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    b->block_threads = best;
    b->rows = best_rows;
    b->tuned = true;
    batch_clear_graphs(b);
    if (block_threads) *block_threads = best;
    if (rows) *rows = best_rows;
    if (st != LBM_OK) return st;
    return batch_join(b, false);
}

lbm_status lbm_batch_tune(lbm_batch* b, int* block_threads, int* rows) {
    NvtxRange range_("lbm_batch_tune");
    if (!b) return LBM_EINVAL;
    lbm_status st = batch_tune_shape(b, block_threads, rows);
    if (st != LBM_OK) return st;
    bool timed = false;  // a batch of AA lattices only: no scheme to choose
    for (auto& g : b->groups) timed = timed || !g.aa;
    if (!timed) return LBM_OK;
    // streaming scheme: a ping-pong group whose lattices could run the AA scheme is timed both
    // ways at the chosen shape; it moves to AA only when that is faster by more than 3 %
    if ((st = batch_upload(b)) != LBM_OK) return st;
    bool moved = false;
    for (auto& g : b->groups) {
        if (!group_aa_eligible(b, g)) continue;
        float pp = 0.0f, aa = 0.0f;
        if ((st = time_group(b, g, false, &pp)) != LBM_OK) return st;
        if ((st = time_group(b, g, true, &aa)) != LBM_OK) return st;
        b->last_pp_ms = pp;
        b->last_aa_ms = aa;
        if (aa < 0.97f * pp) {
            for (int k : g.members)
                if ((st = convert_to_aa(b->ctx[k])) != LBM_OK) return st;
            moved = true;
        }
    }
    if (moved) {
        LBM_BCUDA(cudaStreamSynchronize(b->stream));
        if ((st = batch_group(b)) != LBM_OK) return st;
        batch_clear_graphs(b);
    }
    // launch: a ping-pong group runs each member's own single-lattice kernel where that is more
    // than 3 % faster than the fused launch (lattices that fill the GPU alone, with a kernel
    // that reads its parameters from the constant bank and so takes fewer registers)
    if ((st = batch_upload(b)) != LBM_OK) return st;
    bool changed = false;
    for (auto& g : b->groups) {
        if (g.aa) continue;
        float fused = 0.0f, solo = 0.0f;
        if ((st = time_group(b, g, false, &fused)) != LBM_OK) return st;
        if ((st = time_solo(b, g, &solo)) != LBM_OK) return st;
        const bool want = solo < 0.97f * fused;
        changed = changed || want != g.solo;
        g.solo = want;
    }
    if (changed) batch_clear_graphs(b);
    return batch_join(b, false);
}

lbm_status lbm_batch_set_launch_mode(lbm_batch* b, int mode) {
    if (!b || (mode != LBM_BATCH_FUSED && mode != LBM_BATCH_PER_LATTICE)) return LBM_EINVAL;
    for (auto& g : b->groups)
        if (!g.aa) g.solo = mode == LBM_BATCH_PER_LATTICE;
    batch_clear_graphs(b);
    return LBM_OK;
}

lbm_status lbm_batch_launch_groups(const lbm_batch* b, int* fused, int* per_lattice) {
    if (!b) return LBM_EINVAL;
    int nf = 0, ns = 0;
    for (auto& g : b->groups) (g.solo ? ns : nf) += 1;
    if (fused) *fused = nf;
    if (per_lattice) *per_lattice = ns;
    return LBM_OK;
}

lbm_status lbm_batch_set_scheme(lbm_batch* b, int scheme) {
    if (!b || (scheme != LBM_SCHEME_AA && scheme != LBM_SCHEME_PINGPONG)) return LBM_EINVAL;
    if (scheme == LBM_SCHEME_PINGPONG) return LBM_OK;  // ping-pong members stay as they are
    LBM_BCUDA(cudaSetDevice(b->device));
    lbm_status st = batch_join(b, true);
    if (st != LBM_OK) return st;
    LBM_BCUDA(cudaStreamSynchronize(b->stream));
    bool moved = false;
    for (lbm_ctx* c : b->ctx)
        if (!c->aa && aa_eligible(&c->prm, c->lat)) {
            if ((st = convert_to_aa(c)) != LBM_OK) return st;
            moved = true;
        }
    if (moved) {
        if ((st = batch_group(b)) != LBM_OK) return st;
        batch_clear_graphs(b);
    }
    return batch_join(b, false);
}

lbm_status lbm_batch_scheme_times(const lbm_batch* b, double* pp_ms, double* aa_ms) {
    if (!b) return LBM_EINVAL;
    if (pp_ms) *pp_ms = b->last_pp_ms;
    if (aa_ms) *aa_ms = b->last_aa_ms;
    return LBM_OK;
}

lbm_status lbm_batch_set_block(lbm_batch* b, int block_threads, int rows) {
    if (!b || !(block_threads == 32 || block_threads == 64 || block_threads == 128 ||
                block_threads == 256) || rows < 1 || rows > 64)
        return LBM_EINVAL;
    if (b->block_threads != block_threads || b->rows != rows) batch_clear_graphs(b);
    b->block_threads = block_threads;
    b->rows = rows;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : "null batch"; }

}  // extern "C"

// ---- footprint and serving loop ---------------------------------------------------------------
#include <chrono>
#include <deque>

namespace {

unsigned long long footprint_of(const lbm_params* p, const lbm_lattice& L, int has_phi_field) {
    const unsigned long long ns = (unsigned long long)p->nx * p->ny * p->nz;
    const unsigned long long sq = (ns + 63) / 64 * 64;
    const unsigned long long elem = p->storage == LBM_STORE_FP32 ? 4 : 2;
    const unsigned long long nq = (L.q == 15 ? 15 : lbm::kQ) + lbm::kQT;
    // two population copies (one with the AA scheme)
    unsigned long long b = (L.scheme == LBM_SCHEME_AA ? 1ull : 2ull) * nq * elem * sq;
    if (p->flow_bc[1] == LBM_FLOW_OUTFLOW) b += 2ull * lbm::kOutSlots * 4 * p->ny * p->nz;
    if (p->storage != LBM_STORE_FP32) b += 2ull * 4 * ns;  // temperature planes
    if (has_phi_field) b += 4 * ns;
    b += 9ull * 4 * ns;  // macro fields of the residual
    b += 5ull * 8 * lbm::reduction_blocks() + 8ull * (p->nx > p->ny ? p->nx : p->ny) + 64;
    return b;
}

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct lbm_server {
    struct Req {
        long long id = 0;
        // residual taken in the batched residual launch (D3Q19, halfway walls); the others
        // take lbm_residual's launches
        bool batched_residual = true;
        lbm_params p{};
        double phi = 1.0, K = 0.0, F_phi = 0.0, alpha_m = -1.0, phi_ref = 0.0;
        std::vector<float> phi_field;
        double tol = 1e-6;
        long long max_steps = 1;
        unsigned long long bytes = 0;
        double t_submit = 0.0, t_admit = 0.0;
        lbm_ctx* ctx = nullptr;
        double r_u = HUGE_VAL, r_T = HUGE_VAL;
        float* out_u = nullptr;  // caller's host buffers for the final fields (or NULL)
        float* out_T = nullptr;
        int skipped = 0;  // admission rounds in which later requests were admitted before it
    };
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    unsigned long long budget = 0, used = 0;
    long long max_active_sites = 0;  // 0: no cap
    long long active_sites = 0;
    int policy = LBM_ADMIT_FIFO;
    int chunk = 100;
    std::deque<Req*> queue;
    std::vector<Req*> active;
    std::vector<lbm_result> done;
    lbm_batch* batch = nullptr;
    // block shape of the batched step (0: not tuned yet) and the lattice count of the batch it
    // was tuned on
    int batch_threads = 0, batch_rows = 0;
    size_t tuned_lattices = 0;
    // batched residual of the batched lattices: their table, block map and totals, pinned on
    // the host and on the device, grown as needed
    lbm::ResLattice* h_tab = nullptr;
    lbm::ResLattice* d_tab = nullptr;
    int2* h_blk = nullptr;
    int2* d_blk = nullptr;
    double* h_out = nullptr;
    double* d_out = nullptr;
    size_t tab_cap = 0, blk_cap = 0;
    bool dirty = true;
    long long next_id = 1;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

// Room for n lattices and nblk blocks in the batched-residual buffers.
lbm_status server_reserve(lbm_server* s, size_t n, size_t nblk) {
    if (n > s->tab_cap) {
        const size_t cap = n > 2 * s->tab_cap ? n : 2 * s->tab_cap;
        cudaFreeHost(s->h_tab);
        cudaFree(s->d_tab);
        cudaFreeHost(s->h_out);
        cudaFree(s->d_out);
        s->h_tab = nullptr;
        s->d_tab = nullptr;
        s->h_out = nullptr;
        s->d_out = nullptr;
        s->tab_cap = 0;
        if (cudaHostAlloc(&s->h_tab, cap * sizeof(lbm::ResLattice), cudaHostAllocDefault) != cudaSuccess ||
            cudaMalloc(&s->d_tab, cap * sizeof(lbm::ResLattice)) != cudaSuccess ||
            cudaHostAlloc(&s->h_out, cap * 5 * sizeof(double), cudaHostAllocDefault) != cudaSuccess ||
            cudaMalloc(&s->d_out, cap * 5 * sizeof(double)) != cudaSuccess)
            return LBM_ENOMEM;
        s->tab_cap = cap;
    }
    if (nblk > s->blk_cap) {
        const size_t cap = nblk > 2 * s->blk_cap ? nblk : 2 * s->blk_cap;
        cudaFreeHost(s->h_blk);
        cudaFree(s->d_blk);
        s->h_blk = nullptr;
        s->d_blk = nullptr;
        s->blk_cap = 0;
        if (cudaHostAlloc(&s->h_blk, cap * sizeof(int2), cudaHostAllocDefault) != cudaSuccess ||
            cudaMalloc(&s->d_blk, cap * sizeof(int2)) != cudaSuccess)
            return LBM_ENOMEM;
        s->blk_cap = cap;
    }
    return LBM_OK;
}

void server_finish(lbm_server* s, size_t k, int status) {
    lbm_server::Req* r = s->active[k];
    lbm_result res{};
    res.id = r->id;
    res.status = status;
    res.steps = r->ctx ? r->ctx->steps : 0;
    res.r_u = r->r_u;
    res.r_T = r->r_T;
    res.nu_avg = res.nu_mp = NAN;
    res.mass_dev = res.heat_dev = NAN;
    if (r->ctx && status != LBM_REQ_FAILED) {
        if (r->p.heat_bc[0] == LBM_HEAT_DIRICHLET && r->p.nx >= 2)
            lbm_nusselt(r->ctx, 0, &res.nu_avg, nullptr, &res.nu_mp);
        lbm_sums(r->ctx, &res.mass_dev, &res.heat_dev);
        if (r->out_u || r->out_T) lbm_macros(r->ctx, nullptr, r->out_u, r->out_T);
    }
    res.t_submit = r->t_submit;
    res.t_admit = r->t_admit;
    res.t_done = now_s(s->t0);
    res.bytes = r->bytes;
    res.sites = (long long)r->p.nx * r->p.ny * r->p.nz;
    res.storage = r->p.storage;
    s->done.push_back(res);
    lbm_destroy(r->ctx);
    s->used -= r->bytes;
    s->active_sites -= res.sites;
    delete r;
    s->active.erase(s->active.begin() + (long)k);
    s->dirty = true;
}

}  // namespace

extern "C" {

lbm_status lbm_footprint(const lbm_params* p, int has_phi_field, unsigned long long* bytes) {
    if (!p || !bytes) return LBM_EINVAL;
    lbm_lattice L;
    if (derive(p, &L)) return LBM_EINVAL;
    *bytes = footprint_of(p, L, has_phi_field);
    return LBM_OK;
}

lbm_status lbm_server_create(unsigned long long budget_bytes, int chunk, void* stream,
                             lbm_server** out) {
    if (!out || chunk < 1) return LBM_EINVAL;
    lbm_server* s = new (std::nothrow) lbm_server();
    if (!s) return LBM_ENOMEM;
    s->chunk = chunk;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess && !budget_bytes) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        budget_bytes = (unsigned long long)(0.8 * (double)fr);
    }
    if (e == cudaSuccess) {
        if (stream) {
            s->stream = (cudaStream_t)stream;
        } else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = e == cudaSuccess;
        }
    }
    if (e != cudaSuccess) {
        delete s;
        return LBM_ECUDA;
    }
    s->budget = budget_bytes;
    *out = s;
    return LBM_OK;
}

lbm_status lbm_server_submit(lbm_server* s, const lbm_params* p, const lbm_medium* m, double tol,
                             long long max_steps, long long* id) {
    if (!s || !p || !(tol > 0.0) || max_steps < 1) return LBM_EINVAL;
    lbm_lattice L;
    if (derive(p, &L)) return LBM_EINVAL;
    auto* r = new (std::nothrow) lbm_server::Req();
    if (!r) return LBM_ENOMEM;
    r->p = *p;
    // the AA scheme when asked for; LBM_SCHEME_AUTO is served with two copies
    if (p->scheme != LBM_SCHEME_AA) r->p.scheme = LBM_SCHEME_PINGPONG;
    // a 16-bit format cannot bring the residual below its floor: such a request is stored in
    // FP32, so that it converges at the accuracy it asked for
    if ((p->storage == LBM_STORE_FP16_DEV && tol < LBM_RESIDUAL_FLOOR_FP16) ||
        (p->storage == LBM_STORE_BF16_DEV && tol < LBM_RESIDUAL_FLOOR_BF16))
        r->p.storage = LBM_STORE_FP32;
    if (r->p.scheme == LBM_SCHEME_AA && !aa_eligible(&r->p, L)) {
        delete r;
        return LBM_EINVAL;
    }
    // D3Q15 and node-wall lattices batch, but take their residuals one lattice at a time
    r->batched_residual = L.q == 19 && !L.node_walls;
    if (m) {
        r->phi = m->phi;
        r->K = m->K;
        r->F_phi = m->F_phi;
        r->alpha_m = m->alpha_m;
        r->phi_ref = m->phi_ref;
        if (m->phi_field)
            r->phi_field.assign(m->phi_field, m->phi_field + (size_t)p->nx * p->ny * p->nz);
    }
    r->tol = tol;
    r->max_steps = max_steps;
    r->bytes = footprint_of(&r->p, L, m && m->phi_field ? 1 : 0);
    if (r->bytes > s->budget) {
        delete r;
        return LBM_EINVAL;
    }
    r->id = s->next_id++;
    r->t_submit = now_s(s->t0);
    s->queue.push_back(r);
    if (id) *id = r->id;
    return LBM_OK;
}

lbm_status lbm_server_advance(lbm_server* s, int* n_active, int* n_queued) {
    NvtxRange range_("lbm_server_advance");
    if (!s) return LBM_EINVAL;
    if (cudaSetDevice(s->device) != cudaSuccess) return LBM_ECUDA;
    // admission in arrival order while a request fits the memory budget and, with a cap, the
    // admitted lattices hold fewer sites than the cap (a lone request is always admitted).
    // FIFO stops at the first request that does not fit; BACKFILL lets later requests that fit
    // go ahead of it, until it has been passed over in kMaxSkips rounds.
    constexpr int kMaxSkips = 20;
    bool passed = false;
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        lbm_server::Req* r = *it;
        const long long sites = (long long)r->p.nx * r->p.ny * r->p.nz;
        const bool fits = s->used + r->bytes <= s->budget &&
                          !(s->max_active_sites > 0 && s->active_sites > 0 &&
                            s->active_sites + sites > s->max_active_sites);
        if (!fits) {
            if (s->policy != LBM_ADMIT_BACKFILL) break;
            if (!passed) {  // the oldest waiting request: later ones may pass it ...
                passed = true;
                if (++r->skipped > kMaxSkips) break;  // ... but not for ever
            }
            ++it;
            continue;
        }
        it = s->queue.erase(it);
        s->active_sites += sites;
        r->t_admit = now_s(s->t0);
        lbm_status st = lbm_create(&r->p, s->stream, &r->ctx);
        if (st == LBM_OK)
            st = lbm_set_medium(r->ctx, r->phi_field.empty() ? nullptr : r->phi_field.data(),
                                r->phi, r->K, r->F_phi, r->alpha_m, r->phi_ref);
        s->active.push_back(r);
        s->used += r->bytes;
        s->dirty = true;
        if (st != LBM_OK) server_finish(s, s->active.size() - 1, LBM_REQ_FAILED);
    }
    if (!s->active.empty()) {
        // a lattice of at least kBatchMaxSites sites steps alone (its own step kernel, the
        // paired one where it applies, as dependent launches); the other, smaller ones, whose
        // steps are too short to fill the GPU, advance together in one batched launch per
        // step and kernel variant
        constexpr long long kBatchMaxSites = 512 * 1024;
        auto small = [&](const lbm_server::Req* r) {
            return (long long)r->p.nx * r->p.ny * r->p.nz < kBatchMaxSites;
        };
        if (s->dirty) {
            lbm_batch_destroy(s->batch);
            s->batch = nullptr;
            std::vector<lbm_ctx*> ctxs;
            for (auto* r : s->active)
                if (small(r)) ctxs.push_back(r->ctx);
            if (!ctxs.empty()) {
                lbm_status st = lbm_batch_create(ctxs.data(), (int)ctxs.size(), s->stream, &s->batch);
                if (st != LBM_OK) return st;
                // the block shape: tuned on a batch of at least kTuneMinLattices lattices and
                // again whenever the batch has grown to twice the size it was tuned on (the
                // timed launches leave the state unchanged, the streaming scheme is not
                // changed); every other batch reuses the last shape
                constexpr size_t kTuneMinLattices = 8;
                if (ctxs.size() >= kTuneMinLattices && ctxs.size() >= 2 * s->tuned_lattices) {
                    st = batch_tune_shape(s->batch, &s->batch_threads, &s->batch_rows);
                    s->tuned_lattices = ctxs.size();
                } else if (s->batch_threads > 0) {
                    st = lbm_batch_set_block(s->batch, s->batch_threads, s->batch_rows);
                }
                if (st != LBM_OK) return st;
            }
            s->dirty = false;
        }
        lbm_status st = LBM_OK;
        for (auto* r : s->active)
            if (!small(r) && (st = lbm_step(r->ctx, s->chunk)) != LBM_OK) return st;
        if (s->batch && (st = lbm_batch_step(s->batch, s->chunk)) != LBM_OK) return st;
        // every residual queued behind the chunk, then one synchronisation for all of them:
        // the batched D3Q19 halfway-wall lattices' residuals in one launch per kernel variant
        // (the sums of lbm_residual, bit for bit), the others one lattice at a time
        const size_t na = s->active.size();
        std::vector<lbm_status> launched(na, LBM_OK);
        std::vector<int> slot(na, -1);  // entry in the batched residual's table
        {
            std::vector<std::pair<int, size_t>> items;  // (kernel variant, active index)
            for (size_t k = 0; k < na; ++k) {
                lbm_ctx* c = s->active[k]->ctx;
                if (!small(s->active[k]) || !s->active[k]->batched_residual) continue;
                lbm_status sk = usable(c);
                if (sk == LBM_OK) sk = aa_settle(c);
                if (sk == LBM_OK) sk = ensure_mac(c);
                if (sk != LBM_OK) {
                    launched[k] = sk;
                    continue;
                }
                const int variant = (c->kp.phi_field ? 1 : 0) | (c->outflow ? 2 : 0) |
                                    (c->lat.enthalpy ? 4 : 0) | (c->prm.storage << 3);
                items.emplace_back(variant, k);
            }
            std::stable_sort(items.begin(), items.end(),
                             [](const std::pair<int, size_t>& a, const std::pair<int, size_t>& b) {
                                 return a.first < b.first;
                             });
            size_t nblk = 0;
            for (auto& it : items) nblk += (size_t)lbm::residual_blocks(s->active[it.second]->ctx->ns);
            if (!items.empty()) {
                if ((st = server_reserve(s, items.size(), nblk)) != LBM_OK) return st;
                size_t b = 0, first = 0;  // first: start of the current variant's run
                for (size_t i = 0; i < items.size(); ++i) {
                    lbm_ctx* c = s->active[items[i].second]->ctx;
                    if (items[i].first != items[first].first) first = i;
                    lbm::ResLattice& R = s->h_tab[i];
                    R.p = c->kp;
                    R.pl = c->pl[c->cur];
                    R.cu = c->mac + (size_t)(c->snap ^ 1) * 4 * c->ns;  // new fields
                    R.cT = R.cu + 3 * c->ns;
                    R.pu = c->have_prev ? c->mac + (size_t)c->snap * 4 * c->ns : nullptr;
                    R.pT = R.pu ? R.pu + 3 * c->ns : nullptr;
                    R.partials = c->partials;
                    R.out = s->d_out + 5 * i;
                    R.nr = lbm::residual_blocks(c->ns);
                    R.pad_ = 0;
                    for (int j = 0; j < R.nr; ++j) s->h_blk[b++] = make_int2((int)(i - first), j);
                    slot[items[i].second] = (int)i;
                }
                const size_t n = items.size();
                if (cudaMemcpyAsync(s->d_tab, s->h_tab, n * sizeof(lbm::ResLattice),
                                    cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
                    cudaMemcpyAsync(s->d_blk, s->h_blk, nblk * sizeof(int2), cudaMemcpyHostToDevice,
                                    s->stream) != cudaSuccess)
                    return LBM_ECUDA;
                // one launch per kernel variant, over its run of the table
                size_t i0 = 0, b0 = 0;
                while (i0 < n) {
                    size_t i1 = i0, b1 = b0;
                    while (i1 < n && items[i1].first == items[i0].first) b1 += (size_t)s->h_tab[i1++].nr;
                    lbm_ctx* c = s->active[items[i0].second]->ctx;
                    if (lbm::launch_batch_residual(s->d_tab + i0, s->d_blk + b0, (int)(b1 - b0),
                                                   c->kp.phi_field != nullptr, c->outflow,
                                                   c->prm.storage, c->lat.enthalpy != 0,
                                                   s->stream) != cudaSuccess)
                        return LBM_ECUDA;
                    i0 = i1;
                    b0 = b1;
                }
                if (lbm::launch_batch_residual_finish(s->d_tab, (int)n, s->stream) != cudaSuccess ||
                    cudaMemcpyAsync(s->h_out, s->d_out, n * 5 * sizeof(double),
                                    cudaMemcpyDeviceToHost, s->stream) != cudaSuccess)
                    return LBM_ECUDA;
            }
        }
        for (size_t k = 0; k < na; ++k)
            if (slot[k] < 0 && launched[k] == LBM_OK) launched[k] = residual_launch(s->active[k]->ctx);
        if (cudaStreamSynchronize(s->stream) != cudaSuccess) return LBM_ECUDA;
        std::vector<int> status(na, -1);
        for (size_t k = 0; k < na; ++k) {
            lbm_server::Req* r = s->active[k];
            if (slot[k] >= 0 && launched[k] == LBM_OK)
                std::memcpy(r->ctx->hres, s->h_out + 5 * (size_t)slot[k], 5 * sizeof(double));
            st = launched[k] == LBM_OK ? residual_collect(r->ctx, &r->r_u, &r->r_T) : launched[k];
            if (st == LBM_EUNSTABLE) status[k] = LBM_REQ_UNSTABLE;
            else if (st != LBM_OK) status[k] = LBM_REQ_FAILED;
            else if (r->r_u < r->tol && r->r_T < r->tol) status[k] = LBM_REQ_CONVERGED;
            else if (r->ctx->steps >= r->max_steps) status[k] = LBM_REQ_MAX_STEPS;
        }
        for (size_t k = s->active.size(); k-- > 0;)
            if (status[k] >= 0) server_finish(s, k, status[k]);
    }
    if (s->active.empty() && s->batch) {
        lbm_batch_destroy(s->batch);
        s->batch = nullptr;
    }
    if (n_active) *n_active = (int)s->active.size();
    if (n_queued) *n_queued = (int)s->queue.size();
    return LBM_OK;
}

lbm_status lbm_server_set_policy(lbm_server* s, int policy) {
    if (!s || (policy != LBM_ADMIT_FIFO && policy != LBM_ADMIT_BACKFILL)) return LBM_EINVAL;
    s->policy = policy;
    return LBM_OK;
}

lbm_status lbm_server_set_output(lbm_server* s, long long id, float* u, float* T) {
    if (!s) return LBM_EINVAL;
    for (auto* r : s->queue)
        if (r->id == id) {
            r->out_u = u;
            r->out_T = T;
            return LBM_OK;
        }
    for (auto* r : s->active)
        if (r->id == id) {
            r->out_u = u;
            r->out_T = T;
            return LBM_OK;
        }
    return LBM_EINVAL;  // unknown or already finished
}

lbm_status lbm_server_poll(lbm_server* s, lbm_result* out, int max, int* n) {
    if (!s || (max > 0 && !out)) return LBM_EINVAL;
    int k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.erase(s->done.begin());
    }
    if (n) *n = k;
    return LBM_OK;
}

double lbm_server_clock(const lbm_server* s) { return s ? now_s(s->t0) : 0.0; }

lbm_status lbm_server_set_fill(lbm_server* s, long long max_active_sites) {
    if (!s || max_active_sites < 0) return LBM_EINVAL;
    s->max_active_sites = max_active_sites;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    lbm_batch_destroy(s->batch);
    for (auto* r : s->active) {
        lbm_destroy(r->ctx);
        delete r;
    }
    for (auto* r : s->queue) delete r;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFreeHost(s->h_tab);
    cudaFree(s->d_tab);
    cudaFreeHost(s->h_blk);
    cudaFree(s->d_blk);
    cudaFreeHost(s->h_out);
    cudaFree(s->d_out);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
