/*
 * lbm.h -- C ABI of the GB300 (sm_103a) fused stream-collide library for the 3D
 * double-distribution-function MRT lattice Boltzmann model of convection heat transfer in
 * porous media at the REV scale (Liu & He, arXiv:1611.03329).
 *
 * One time step advances, at every lattice site, the D3Q19 MRT density populations f
 * (Sec. 3.1.2, Eqs. 8-11 and 19-28, generalized non-Darcy force of Eq. 4) and the D3Q7 MRT
 * temperature populations g (Sec. 3.2, Eqs. 33-43), streaming in pull form (Eqs. 10, 35)
 * with halfway bounce-back walls, velocity inlets, anti-bounce-back Dirichlet walls and an
 * anchored convective outflow.
 *
 * Conventions shared by every call:
 *  - Every call returns an lbm_status; nothing throws across the ABI.  A CUDA failure and a
 *    timed-out device wait are sticky: once a call returns LBM_ECUDA or LBM_ETIMEOUT the
 *    context only accepts lbm_destroy, lbm_last_error and lbm_status_string.
 *  - Field arrays are x-fastest: site s = x + nx*(y + ny*z); population arrays are
 *    q-major, f[i*ns + s] with ns = nx*ny*nz and the velocity order of Eq. 19 (D3Q19) and
 *    of the first seven columns of Eq. 12 (D3Q7).  Vector fields are [3][ns].
 *  - "host" pointers are caller-owned CPU memory (pinned or pageable); the library copies
 *    from or into them and keeps no reference.  "device" pointers are caller-owned GPU
 *    memory on the context's device.  The context owns all of its own device memory.
 *  - Work is queued on the stream given to lbm_create.  Calls that return results to host
 *    memory synchronise that stream; lbm_step and the *_device calls do not.
 *  - A context is not thread-safe; use one context per host thread or serialise.
 *  - Faces are numbered x-low, x-high, y-low, y-high, z-low, z-high (0..5).
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,    /* an argument or parameter is out of range; nothing was changed */
    LBM_ENOMEM = 2,    /* device allocation failed; the context is unusable */
    LBM_ECUDA = 3,     /* a CUDA call failed (sticky, see lbm_last_error) */
    LBM_EUNSTABLE = 4, /* a reduction found NaN or Inf in the state */
    LBM_ESTATE = 5,    /* call not allowed in the context's current state */
    LBM_ETIMEOUT = 6   /* a bounded device-side wait ran out and the step stopped early
                          (sticky, see LBM_KERNEL_TMA) */
} lbm_status;

/* Flow boundary kinds (per face). */
enum {
    LBM_FLOW_PERIODIC = 0, /* both faces of the axis must be periodic */
    LBM_FLOW_WALL = 1,     /* resting no-slip wall, halfway bounce-back */
    LBM_FLOW_VELOCITY = 2, /* moving wall / velocity inlet with face_u (bounce-back) */
    LBM_FLOW_OUTFLOW = 3,  /* convective outflow; x-high face only */
    LBM_FLOW_NEE = 4       /* node wall by non-equilibrium extrapolation (see below) */
};

/* Thermal boundary kinds (per face). */
enum {
    LBM_HEAT_PERIODIC = 0,  /* must match a periodic flow face */
    LBM_HEAT_ADIABATIC = 1, /* zero heat flux, bounce-back of g */
    LBM_HEAT_DIRICHLET = 2, /* wall temperature face_T, anti-bounce-back of g */
    LBM_HEAT_OUTFLOW = 3,   /* convective outflow; only on an outflow face */
    LBM_HEAT_NEE_DIRICHLET = 4, /* node wall at face_T (with LBM_FLOW_NEE) */
    LBM_HEAT_NEE_ADIABATIC = 5  /* node wall at the temperature of the fluid beside it */
};
/* Node walls (the paper's boundary scheme, non-equilibrium extrapolation [50], Sec. 4): the
 * layer of sites on an LBM_FLOW_NEE face is the wall, moving at face_u; its temperature is
 * face_T (LBM_HEAT_NEE_DIRICHLET) or that of the fluid beside it (LBM_HEAT_NEE_ADIABATIC).  A
 * wall site does not stream: with x_f the fluid site beside it (plus the inward normal of
 * every node-wall face it lies on), its populations are the wall equilibrium plus the
 * streamed non-equilibrium part of x_f, f = f_eq(rho_b, u_w) + [f(x_f) - f_eq(rho_f, u_f)]
 * and g = g_eq(T_b, u_w) + [g(x_f) - g_eq(T_f, u_f)], collided at its own state with the
 * velocity prescribed as u_w (rho_b = rho_f, or rho0 on a wall that withdraws fluid).  The
 * walls sit on the sites, so a channel of ny sites has height ny - 1 (give L).  FP32 storage,
 * no outflow face, no enthalpy model, outside lbm_batch / lbm_server; >= 3 sites across. */

/* Mapping from the dimensionless problem statement to lattice units. */
enum {
    LBM_MAP_CAVITY = 0,  /* natural convection, Eq. 56 (Ra, Pr, Ma, J, sigma, Gamma) */
    LBM_MAP_CHANNEL = 1, /* mixed convection, Eq. 51 (Re, u0, Pr, J, sigma, Gamma, Ri) */
    LBM_MAP_LATTICE = 2  /* lattice units given directly (nu_e, alpha_f, gbeta) */
};

/* Storage of the populations (arithmetic is FP32 in every case).  Bytes per site are those a
 * time step reads and writes (each population once each way):
 *  LBM_STORE_FP32     : FP32 deviations f_i - w_i rho0 and g_i - omega_i sigma T0 (208 B/site;
 *                       D3Q15: 176 B/site);
 *  LBM_STORE_FP16_DEV : FP16 scaled deviations, rounded to nearest: 64 (f_i - w_i rho0) for the
 *                       D3Q19 planes (a power of two: the kernels convert without multiplying
 *                       and collide in these units), and
 *                       for the D3Q7 planes (g_i - omega_i sigma T_x) / omega_i against the
 *                       site's own temperature T_x, whose deviation T_x - T0 is kept in an FP32
 *                       temperature plane (26 x 2 B + 4 B, read and written: 112 B/site);
 *  LBM_STORE_BF16_DEV : the same in BF16 (112 B/site).
 * A porosity field (lbm_set_medium) adds 4 B/site read. */
enum { LBM_STORE_FP32 = 0, LBM_STORE_FP16_DEV = 1, LBM_STORE_BF16_DEV = 2 };

/*
 * Problem statement (Sec. 2, Eqs. 1-7, and the problem setups of Sec. 4).  Fill it with
 * lbm_params_default() first; every field then holds the paper's default.
 */
typedef struct lbm_params {
    int nx, ny, nz;  /* lattice sites per axis, each >= 1 (>= 3 along x with an outflow) */
    int storage;     /* LBM_STORE_* */
    int mapping;     /* LBM_MAP_* */
    double L;        /* characteristic length in lattice units; <= 0: nx (cavity,
                        lattice) or ny (channel) -- the halfway walls make L = N */
    double Ra, Da, Pr, J, sigma, Gamma, Ma; /* Eq. 7 and Eq. 56 (Ma = u_c / c_s) */
    double Re, Ri, u0;                      /* channel: Eq. 51 with u1 = u0, H = L */
    double dT;                              /* T_h - T_c (1) */
    double T0, rho0, varpi;                 /* reference temperature (0.5), mean density
                                               (1), D3Q7 parameter varpi in (0,1) (0.5) */
    /* free relaxation rates of Sec. 4 (defaults 1.1, 1.1, 1.1, 1.1, 1.2, 1, 1.2, 1.2) */
    double s_e, s_eps, s_q, s_pi, s_m, zeta_T, zeta_e, zeta_nu;
    double nu_e, alpha_f, gbeta;     /* LBM_MAP_LATTICE: effective viscosity, fluid
                                        diffusivity (<= 0: nu/Pr) and g*beta */
    int gravity_axis;                /* 0, 1, 2 (z, Sec. 4.2) */
    int gravity_sign;                /* -1: gravity points to -axis (hot fluid rises) */
    double accel[3];                 /* external acceleration a of Eq. 5 */
    int flow_bc[6];                  /* LBM_FLOW_* per face */
    int heat_bc[6];                  /* LBM_HEAT_* per face */
    double face_T[6];                /* Dirichlet wall temperatures */
    double face_u[6][3];             /* velocity of LBM_FLOW_VELOCITY faces */
    double T_init;                   /* initial uniform temperature */
    double U_out;                    /* convective outflow speed; <= 0: u0 */
    /* enthalpy-based D3Q7 model for solid-liquid phase change (App. B); FP32 storage,
     * uniform medium and no outflow only.  The D3Q7 populations then carry the effective
     * enthalpy En_e (Eq. B7); T and the liquid fraction follow Eqs. B8-B9; the flow is
     * collided only where f_l >= 0.5 (elsewhere it rests at f_eq(rho, 0), u = 0). */
    int enthalpy;                    /* 1 enables the model */
    int flow_off;                    /* 1: u = 0 everywhere (conduction melting) */
    double T_m;                      /* melting point; T_s = T_l = T_m unless T_l > T_s */
    double T_s, T_l;                 /* solidus and liquidus temperatures */
    double St;                       /* Stefan number c_pl dT / L_a (1) */
    double c_pl, c_ps;               /* specific heats (1, 1); c_ref = harmonic mean (Eq. B13) */
    double sigma_s, sigma_l;         /* heat-capacity ratios (Eq. B4); <= 0: sigma */
    double alpha_ratio;              /* alpha_l / alpha_s (1); alpha_l = the fluid diffusivity */
    /* flow lattice: 19 (D3Q19-MRT, Sec. 3.1.2, the default; 0 reads as 19) or 15 (D3Q15-MRT,
     * Sec. 3.1.1: velocities of Eq. 12, moments of Eq. 13 / Eq. A1, equilibria of Eq. 15,
     * Lambda of Eq. 16 from s_e, s_eps, s_q, s_nu, s_m, forcing of Eq. 17).  D3Q15 runs with
     * FP32 storage, without the enthalpy model, and outside lbm_batch / lbm_server; its f
     * arrays in lbm_set_populations / lbm_get_populations hold 15 planes. */
    int q_flow;
    /* population scheme: LBM_SCHEME_PINGPONG (0, the default), LBM_SCHEME_AA or
     * LBM_SCHEME_AUTO, see below */
    int scheme;
    /* LBM_SCHEME_AUTO: cap, in bytes, on the free device memory that lbm_create counts when
     * it chooses the scheme (0, the default: no cap) */
    unsigned long long auto_mem_limit;
} lbm_params;

/* Population schemes.  Both compute the same site update and give bit-identical populations.
 *  LBM_SCHEME_PINGPONG : two copies of the populations; every step pulls from one copy and
 *                        writes the other.
 *  LBM_SCHEME_AA       : one copy, updated in place by alternating two kinds of step: a pull
 *                        step that gathers like ping-pong and pushes each post-collision
 *                        population to the plane the next step reads it from, and a local step
 *                        that reads and writes its own site only.  Half the population memory,
 *                        the same bytes moved per step.  Needs FP32 storage, the D3Q19 lattice,
 *                        no outflow face, no node walls and no enthalpy model; such contexts
 *                        run with LBM_KERNEL_PLAIN, in lbm_batch (their own groups) but not in
 *                        lbm_server.  After an
 *                        odd number of steps, the first call that reads the state (populations,
 *                        macros, Nusselt, sums, residual) first rearranges the copy (a pure
 *                        permutation, no arithmetic) into the layout a pull step reads.
 *  LBM_SCHEME_AUTO     : ping-pong while its footprint fits in the device memory free at
 *                        lbm_create (lbm_params.auto_mem_limit, when above 0, caps that
 *                        figure), else AA where the lattice allows it; lbm_derive_lattice
 *                        reports ping-pong for it; lbm_server runs ping-pong.  The scheme in
 *                        use is lbm_lattice.scheme (lbm_get_lattice). */
#define LBM_SCHEME_PINGPONG 0
#define LBM_SCHEME_AA 1
#define LBM_SCHEME_AUTO 2

/*
 * Lattice-unit parameters derived from an lbm_params (Eq. 32, Eq. 41, Eq. 51 or Eq. 56,
 * Eq. 7) and the medium.  Read-only view for checks and logging.
 */
typedef struct lbm_lattice {
    int nx, ny, nz;
    double L, rho0, T0, sigma, varpi, dT;
    double s[19];              /* diagonal of Lambda in the moment order of Eq. 20 (Eq. 22) */
    double zeta_T, zeta_e, zeta_nu, zeta_alpha; /* Q of Eq. 38 (zeta_alpha of a uniform
                                                   medium; per site with alpha_m >= 0) */
    double s_nu, nu_e, nu, alpha_f, alpha_m, Gamma;
    double gbeta, buoy[3], accel[3];   /* G = buoy (T - T0) + accel */
    double phi, K, F_phi, phi_ref;     /* F_phi < 0: Ergun per site; K may be +inf */
    int has_phi_field;
    double U_out;
    int enthalpy, flow_off;
    double c_pl, c_ref, sigma_s, sigma_l, T_s, T_l, L_a, alpha_s, alpha_l;
    int node_walls;            /* 1 if a face is a node wall (LBM_FLOW_NEE) */
    int q;                     /* flow lattice (19 or 15); with 15, s[] keeps the D3Q19 order
                                  and the D3Q15 rates s_e, s_eps, s_q, s_nu, s_m of Eq. 16 are
                                  s[1], s[2], s[4], s[9], s[16] */
    int scheme;                /* the scheme in use: LBM_SCHEME_PINGPONG or LBM_SCHEME_AA */
} lbm_lattice;

/* Fill p with the paper's defaults (Sec. 4: rho0 = 1, J = sigma = Gamma = 1, varpi = 1/2,
 * the free relaxation rates above, Ma = 0.1, Pr = 1, T0 = 0.5, gravity -z) and all faces
 * periodic.  Host only; never fails for a non-NULL p. */
lbm_status lbm_params_default(lbm_params* p);

/* Derive the lattice parameters of p without creating a context (host only, no GPU):
 * Eq. 56 (cavity) or Eq. 51 read with 1/s_nu (channel) for s_nu, Eq. 32 for nu_e,
 * nu = nu_e / J, alpha_f = nu / Pr, Eq. 41 for zeta_alpha, g beta from u_c = Ma c_s =
 * sqrt(g beta dT L) (cavity) or Ri = g beta dT L / u0^2 (channel).  The medium is the
 * default one (phi = 1, K = Da L^2 or +inf, F_phi = 0).  LBM_EINVAL on any invalid field. */
lbm_status lbm_derive_lattice(const lbm_params* p, lbm_lattice* out);

/* Create a context on the device of `stream` (a cudaStream_t; NULL: the calling thread's
 * current device and a private non-blocking stream), queue its work on that stream,
 * allocate the two population
 * copies and initialise f = f_eq(rho0, u = 0), g = g_eq(T_init, u = 0) (Eqs. 24, 42).
 * The medium starts as phi = 1, K = Da L^2 (Da > 0) or +inf, F_phi = 0.
 * Errors: LBM_EINVAL (invalid params; *out untouched), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(const lbm_params* p, void* stream, lbm_ctx** out);

/* Release all device memory of the context (and its private stream).  NULL is a no-op. */
void lbm_destroy(lbm_ctx* ctx);

/* Porous medium (Eq. 4, Eq. 6, Sec. 2).
 *  phi_field : host, ns floats in (0,1), or NULL for the uniform porosity `phi` in (0,1].
 *  K         : permeability; <= 0 selects Da L^2 (Eq. 7), +inf removes the Darcy and
 *              Forchheimer drag.  With a field, K is the permeability at porosity phi_ref
 *              and K(x) follows Kozeny-Carman, K ~ phi^3 / (1 - phi)^2 (Eq. 6).
 *  F_phi     : Forchheimer inertia coefficient; < 0 selects Ergun's 1.75/sqrt(150 phi^3)
 *              (Eq. 6, per site with a field); 0 is the Brinkman-extended Darcy model.
 *  alpha_m   : matrix thermal diffusivity; < 0 keeps alpha_e = Gamma alpha_f, otherwise
 *              alpha_e(x) = phi alpha_f + (1 - phi) alpha_m and zeta_alpha follows Eq. 41
 *              per site.
 *  phi_ref   : <= 0 selects the mean of phi_field (or phi).
 * Takes effect from the next lbm_step; the populations are not touched.  Synchronises the
 * stream.  Errors: LBM_EINVAL (out-of-range value; nothing changed), LBM_ECUDA. */
lbm_status lbm_set_medium(lbm_ctx* ctx, const float* phi_field, double phi, double K,
                          double F_phi, double alpha_m, double phi_ref);

/* Advance nsteps >= 0 time steps: per site, pull streaming with the boundary rules
 * (Eqs. 10, 35), T from Eq. 39, G from Eq. 5, u from Eqs. 27-28, F from Eq. 4, the D3Q19
 * MRT collision with forcing in moment space (Eqs. 9, 21-23) and the D3Q7 MRT collision
 * (Eqs. 34, 37-38, 43).  Asynchronous on the context's stream; launch errors are returned,
 * execution errors surface at the next synchronising call.  LBM_EINVAL for nsteps < 0. */
lbm_status lbm_step(lbm_ctx* ctx, int nsteps);

/* Step kernels.  Both compute the same site update (Eqs. 9-10, 34-35 with the boundary rules
 * of lbm_step) and give bit-identical populations; they differ in how the streamed
 * populations reach the collision.
 *  LBM_KERNEL_PLAIN : one thread per site, each pull a load through the L1.
 *  LBM_KERNEL_TMA   : persistent blocks over tiles of 64 x 4 sites of one z-plane; for
 *                     tiles inside the y and z ranges the Tensor Memory Accelerator copies,
 *                     a few tiles ahead, one box per population plane (shifted by -e_i) into
 *                     shared memory.  Needs the D3Q19 lattice, nx % 64 == 0, ny >= 4, no node
 *                     walls and no enthalpy model.  A staged load that does not complete within
 *                     one second stops the step early; the next call that synchronises the
 *                     context's stream (lbm_sync, lbm_macros, lbm_residual, lbm_sums,
 *                     lbm_nusselt, lbm_get_populations, ...) then returns LBM_ETIMEOUT
 *                     (sticky).  lbm_test_tma_extra_wait exercises that path.
 *  LBM_KERNEL_PAIRED : one thread per pair of x-adjacent sites; planes whose velocity has
 *                     e_x = 0 are read and written as aligned 2-element accesses and the
 *                     collision runs on the paired FP32 instructions of sm_100 (two sites per
 *                     instruction).  Needs the D3Q19 lattice, the ping-pong scheme, an even
 *                     nx, fewer than ~82 M sites, no node walls and no enthalpy model.
 * lbm_create selects LBM_KERNEL_PAIRED where it applies, else LBM_KERNEL_PLAIN. */
#define LBM_KERNEL_PLAIN 0
#define LBM_KERNEL_TMA 1
#define LBM_KERNEL_PAIRED 2

/* Select the step kernel used by later lbm_step calls.  Prepares the kernel (tensor maps of
 * both population copies, shared-memory limit, a 4-byte device flag owned by ctx).
 * Errors: LBM_EINVAL (unknown kernel, or a lattice the kernel does not take; the selection is
 * unchanged), LBM_ECUDA. */
lbm_status lbm_set_step_kernel(lbm_ctx* ctx, int kernel);

/* The context's step kernel (LBM_KERNEL_*), -1 for ctx == NULL. */
int lbm_get_step_kernel(const lbm_ctx* ctx);

/* Launch settings of the context's single-lattice site kernels, for measurements:
 *  block_threads    : threads per block, 32, 64 (the default), 128 or 256; 0 keeps the
 *                     current value;
 *  dependent_launch : 1 (the default) launches each step kernel as a programmatic dependent
 *                     launch (its blocks may be scheduled while the previous step drains; they
 *                     wait for it before their first load), 0 as an ordinary launch, -1 keeps
 *                     the current setting.
 * Results do not depend on either.  Errors: LBM_EINVAL (a value out of range; nothing changed). */
lbm_status lbm_set_launch(lbm_ctx* ctx, int block_threads, int dependent_launch);

/* Bounds-checked build (the library compiled with -DLBM_BOUNDS_CHECK, e.g.
 * `python -m paper_1611_03329_gb300.build --checked`, liblbm_gb300_checked.so): every site
 * index of a population, temperature-plane, porosity or outflow-history access of the site
 * kernels (step, paired, batched, AA, macros) is checked; an index out of range is replaced by
 * 0 and the first one met is kept.  *first_bad receives it (-1: none) for the current device.
 * The ordinary build returns LBM_EINVAL (nothing is checked there). */
lbm_status lbm_bounds_report(long long* first_bad);

/* TEST ONLY: makes every pipeline stage of the TMA step kernel wait for `bytes` (0 .. 4096)
 * more than its loads bring, so that its bounded waits run out and the failure path of
 * LBM_KERNEL_TMA can be exercised without a fault; 0 (the default) turns it off.  Takes effect
 * from the next lbm_step with LBM_KERNEL_TMA.  Errors: LBM_EINVAL for bytes out of range. */
lbm_status lbm_test_tma_extra_wait(lbm_ctx* ctx, int bytes);

/* Re-initialise the state to equilibrium (Eqs. 24 and 42) with rho = rho0 and, per site,
 * T from T_field (host, ns doubles; NULL: T_uniform) and u from u_field (host, 3 x ns
 * doubles; NULL: 0), using the current medium.  Resets the step counter.  Synchronises. */
lbm_status lbm_init_equilibrium(lbm_ctx* ctx, const double* T_field, const double* u_field,
                                double T_uniform);

/* Replace the stored post-collision populations f*(x, t-1), g*(x, t-1) (host, Q x ns and
 * 7 x ns doubles with Q = 19 or 15 the flow lattice, full values, not deviations).  The outflow history is reset to the
 * stored populations of the x-high column.  Synchronises. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f, const double* g);

/* Copy the stored post-collision populations to host (Q x ns and 7 x ns doubles, Q = 19 or
 * 15, full values); either pointer may be NULL.  Synchronises. */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, double* g);

/* Raw state I/O (checkpoint / restart, and a lossless host round trip of the state).  The
 * state blob holds a 128-byte header (magic "LBMSTATE", version, the lattice extents, flow
 * lattice, storage format, scheme and step count) followed by the populations of the current
 * copy exactly as stored (the Q + 7 planes of sq = ceil(ns / 64) * 64 elements each, in the
 * storage format, FP32 deviations or 16-bit scaled deviations), the FP32 temperature plane of
 * the 16-bit formats (ns floats) and the outflow history (6 x ny x nz floats) when the
 * lattice has them.  lbm_state_bytes gives its size.  No conversion runs on either side: one
 * asynchronous copy per region on the context's stream.  The host buffer (pinned memory
 * gives full copy bandwidth) must stay valid and unchanged until the next synchronising call.
 * lbm_load_state accepts only a blob of a context with the same extents, flow lattice,
 * storage format and scheme (LBM_EINVAL otherwise, nothing changed); it restores the step
 * count.  The parameters and the medium (lbm_set_medium) are not in the blob: a restart
 * context is created from the same lbm_params and given the same medium.  An AA context saves
 * after rearranging an odd-step copy (see LBM_SCHEME_AA).  Errors: LBM_EINVAL (NULL or short
 * buffer, a foreign or truncated blob; nothing changed), LBM_ECUDA. */
lbm_status lbm_state_bytes(const lbm_ctx* ctx, unsigned long long* bytes);
lbm_status lbm_save_state(lbm_ctx* ctx, void* host, unsigned long long bytes);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* host, unsigned long long bytes);

/* Macroscopic fields at the current time, computed from the streamed populations exactly
 * as the step does: rho (Eq. 25), u (Eqs. 27-28), T (Eq. 39).  Host pointers: rho and T
 * ns floats, u 3 x ns floats; any may be NULL.  Synchronises. */
lbm_status lbm_macros(lbm_ctx* ctx, float* rho, float* u, float* T);

/* Same as lbm_macros into device pointers; asynchronous on the context's stream. */
lbm_status lbm_macros_device(lbm_ctx* ctx, float* rho, float* u, float* T);

/* Wall Nusselt numbers of Eqs. 53-55 on a Dirichlet face: -d(theta)/dn at the halfway wall
 * from the quadratic through the wall value and the first two nodes,
 * Nu_local = L (8 T_w - 9 T_0 + T_1) / (3 dT) (positive = heat into the fluid); on a node
 * wall (LBM_HEAT_NEE_DIRICHLET) the second-order one-sided gradient over the wall site and
 * the next two, Nu_local = L (3 T_w - 4 T_1 + T_2) / (2 dT); averaged
 * over the second tangential axis into the profile along the first one (y for x-faces,
 * x otherwise; Eq. 54), whose mean is Nu_3D (Eq. 55) and whose centre value is Nu_mp.
 * FP64 accumulation on the device.  nu_avg, nu_profile (host, length of the first
 * tangential axis) and nu_mp may each be NULL.  Synchronises.
 * Errors: LBM_EINVAL (face not Dirichlet or too few sites normal to it), LBM_EUNSTABLE. */
lbm_status lbm_nusselt(lbm_ctx* ctx, int face, double* nu_avg, double* nu_profile,
                       double* nu_mp);

/* Totals of the stored populations, FP64 accumulation: mass_dev = sum_s sum_i f_i - ns rho0
 * (mass, Eq. 25) and heat_dev = sum_s sum_i g_i - ns sigma T0 (heat, Eq. 39); with the
 * enthalpy model heat_dev is the total effective enthalpy sum_s sum_i g_i (Eq. B7).
 * Either pointer may be NULL.  Synchronises.  LBM_EUNSTABLE if a total is not finite. */
lbm_status lbm_sums(lbm_ctx* ctx, double* mass_dev, double* heat_dev);

/* Steady-state residual: r_u = ||u - u_prev||_2 / ||u||_2 and the same for T, against the
 * fields saved by the previous call (FP64 accumulation); 0 for a field that is zero and
 * unchanged; the first call after create or init returns +inf.  Synchronises.
 * LBM_EUNSTABLE if a field holds NaN or Inf. */
lbm_status lbm_residual(lbm_ctx* ctx, double* r_u, double* r_T);

/* Largest field, in sites, that lbm_residual_noalloc accepts (2^25, e.g. 256 x 256 x 512). */
#define LBM_NOALLOC_MAX_SITES 33554432LL

/* Allocation-free steady-state residual.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- an application that gives the
 * library a fixed arena and forbids cudaMalloc after start-up, or a loop in which an
 * allocation (which may synchronise the device) would stall.
 * It computes what lbm_residual computes, r_u = ||u - u_prev||_2 / ||u||_2 and the same for
 * T (FP64 accumulation), from fields the caller holds, e.g. two results of
 * lbm_macros_device:
 *  u, u_prev : device, 3 x ns floats ([3][ns]);  T, T_prev : device, ns floats;
 *  ns        : 1 .. LBM_NOALLOC_MAX_SITES, else LBM_EINVAL and nothing is launched;
 *  out       : device, 3 doubles, written asynchronously: r_u, r_T (0 for a field that is
 *              zero and unchanged, +inf for one that is zero after changing) and the number
 *              of non-finite values met; when that number is above 0, r_u and r_T are NaN
 *              (a blown-up field never passes a test r < tol);
 *  stream    : cudaStream_t to queue on (NULL: the current device's default stream).
 * The call runs on the stream's device and leaves the calling thread's current device as it
 * found it.  Each of its two launches is checked through its own return code; an error left
 * on the thread by an earlier call is neither reported nor cleared.
 * It allocates nothing: its partial sums live in a static 320 KiB device array that every
 * GPU loading the library holds until exit.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress), so make that first call on each device
 * before any stream capture begins.  All calls share the array: calls whose
 * kernels overlap on the GPU race and must be serialised.  Errors: LBM_EINVAL (NULL pointer or ns out of range), LBM_ECUDA. */
lbm_status lbm_residual_noalloc(const float* u, const float* T, const float* u_prev,
                                const float* T_prev, long long ns, double* out, void* stream);

/* ---- batched launches -----------------------------------------------------------------
 * A batch advances many independent lattices (contexts) with one fused launch per time step
 * and kernel variant (storage format, uniform or field medium, outflow or not, D3Q19 or D3Q15
 * flow lattice, halfway or node walls, ping-pong or AA scheme; an AA lattice takes its own
 * pull or local step in the shared launch): the step of
 * Sec. 3 at every site of every lattice, exactly as lbm_step computes it, so a lattice's
 * results are identical alone and in a batch.  Multi-step sequences are recorded once per
 * step count as a CUDA graph and replayed.  The contexts keep owning their state; after
 * lbm_batch_step every per-context call (macros, Nusselt, sums, ...) sees the new state. */
typedef struct lbm_batch lbm_batch;

/* Group n contexts (same device, each at most once) into a batch queued on `stream`
 * (NULL: a private stream).  The batch reads each context's parameters, medium and state
 * at every lbm_batch_step, so changes made through the contexts are picked up.
 * Errors: LBM_EINVAL (bad list, mixed devices, a failed context), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int n, void* stream, lbm_batch** out);

/* Advance every lattice of the batch by nsteps >= 0 time steps (asynchronous; ordered after
 * and before the contexts' own streams). */
lbm_status lbm_batch_step(lbm_batch* b, int nsteps);

/* Autotuner of the batched step.  (1) Block shape: time the step at 32, 64, 128 and 256
 * threads per block and 1, 2 and 4 z-planes per block and keep the fastest (written to
 * *block_threads and *rows when non-NULL); the timed launches write only the buffers that the
 * next step overwrites, so the lattices' state is unchanged.  AA lattices, updated in place,
 * are not timed, and a batch of AA lattices only takes 32 threads x 4 planes (measured fastest
 * for them).  (2) Streaming scheme: every group of ping-pong lattices that could run the AA
 * scheme is timed both ways at the chosen shape -- AA on scratch, each lattice's second copy
 * filled with its state and stepped in place -- and moves to AA (lbm_batch_set_scheme) only if
 * that is more than 3 % faster (lbm_batch_scheme_times reports the last trial).  (3) Launch:
 * every ping-pong group is timed fused and per lattice (lbm_batch_set_launch_mode), without
 * changing the state, and runs per lattice where that is more than 3 % faster.
 * Synchronises. */
lbm_status lbm_batch_tune(lbm_batch* b, int* block_threads, int* rows);

/* Move every ping-pong member that can run the AA scheme (FP32, D3Q19, no outflow face, no
 * node walls, no enthalpy model) to it: its current copy is permuted into its second copy,
 * which becomes the only one, and the first is freed -- half the population memory, the same
 * populations, bit-identical later steps.  LBM_SCHEME_PINGPONG is accepted and changes
 * nothing (AA members are not moved back).  Synchronises.  LBM_EINVAL for another scheme. */
lbm_status lbm_batch_set_scheme(lbm_batch* b, int scheme);

/* Milliseconds per step of the last group the tuner timed both ways (0 before any trial). */
lbm_status lbm_batch_scheme_times(const lbm_batch* b, double* pp_ms, double* aa_ms);

/* How a batch group's lattices are stepped.  LBM_BATCH_FUSED: one launch per step for all of
 * them (replayed from a graph).  LBM_BATCH_PER_LATTICE: each lattice's own single-lattice step
 * kernel, launched directly, one launch per lattice and step -- faster for lattices that fill
 * the GPU alone, whose kernel then reads its parameters from the constant bank and takes fewer
 * registers.  Results are the same either way.  lbm_batch_tune (stage 3) times both for every
 * ping-pong group and keeps the per-lattice launch where it is more than 3 % faster;
 * lbm_batch_set_launch_mode sets every ping-pong group (AA groups are always fused). */
enum { LBM_BATCH_FUSED = 0, LBM_BATCH_PER_LATTICE = 1 };
lbm_status lbm_batch_set_launch_mode(lbm_batch* b, int mode);
/* Number of groups stepped by the fused launch and per lattice. */
lbm_status lbm_batch_launch_groups(const lbm_batch* b, int* fused, int* per_lattice);

/* Set the block shape of the batched step: threads (32, 64, 128 or 256) and z-planes per
 * block (1..64). */
lbm_status lbm_batch_set_block(lbm_batch* b, int block_threads, int rows);

/* Text of the batch's last error (never NULL). */
const char* lbm_batch_last_error(const lbm_batch* b);

/* Release the batch (not its contexts).  NULL is a no-op. */
void lbm_batch_destroy(lbm_batch* b);

/* Device bytes a context for p will hold, including the residual buffers a solve to steady
 * state allocates (host only, no GPU).  LBM_EINVAL for invalid params. */
lbm_status lbm_footprint(const lbm_params* p, int has_phi_field, unsigned long long* bytes);

/* ---- serving loop ------------------------------------------------------------------------
 * A server takes solve requests as they arrive, admits them in arrival order while their
 * device footprint fits its memory budget, keeps their populations resident and advances all
 * admitted lattices together in chunks of `chunk` steps: lattices below 512 K sites in one
 * batched launch per step (lbm_batch_*), larger ones, which fill the GPU on their own, with
 * their own step kernel (lbm_step), all queued on the server's stream.  The block shape of the
 * batched step is tuned (as stage (1) of lbm_batch_tune, leaving the state unchanged) on the
 * first batch of at least 8 lattices and again whenever a batch has twice the lattices of the
 * one last tuned; other batches reuse the last shape.
 * After every chunk each lattice's steady-state residual (lbm_residual; one synchronisation of
 * the server's stream for all of them) is checked; a request
 * finishes when both residuals fall below its tolerance, when it reaches its step limit, or
 * when its state stops being finite, and its memory is released for the next request.  A
 * request's result depends only on its own problem: it is the same alone and in the mix. */
typedef struct lbm_server lbm_server;

/* Medium of a request (the arguments of lbm_set_medium); phi_field is copied at submit. */
typedef struct lbm_medium {
    const float* phi_field; /* host, ns floats, or NULL */
    double phi, K, F_phi, alpha_m, phi_ref;
} lbm_medium;

enum { LBM_REQ_CONVERGED = 0, LBM_REQ_MAX_STEPS = 1, LBM_REQ_UNSTABLE = 2, LBM_REQ_FAILED = 3 };

/* Residual floors of the 16-bit formats: the rounding of the stored deviations keeps the
 * steady-state residual of a 16-bit solve above about these values (measured on the porous
 * cavities of the precision sweep: FP16 0.8e-4 .. 1.4e-4 in u, BF16 0.7e-3 .. 1.1e-3).  A request
 * whose tolerance lies below the floor of its storage format is served in FP32 storage
 * (lbm_result.storage), so that it can converge at the accuracy it asks for. */
#define LBM_RESIDUAL_FLOOR_FP16 2e-4
#define LBM_RESIDUAL_FLOOR_BF16 2e-3

/* Admission policies (lbm_server_set_policy).  FIFO: requests are admitted strictly in
 * arrival order; the first one that does not fit (memory budget or fill cap) stops admission.
 * BACKFILL: later requests that fit may be admitted ahead of one that does not, until that
 * one has waited 20 rounds with others passing it; then admission is FIFO again until it is in. */
enum { LBM_ADMIT_FIFO = 0, LBM_ADMIT_BACKFILL = 1 };

/* Result of a finished request.  Times are seconds on the server's host clock since
 * lbm_server_create: submitted, admitted (state allocated), finished. */
typedef struct lbm_result {
    long long id;
    int status;                 /* LBM_REQ_* */
    long long steps;            /* time steps taken */
    double r_u, r_T;            /* last residuals */
    double nu_avg, nu_mp;       /* Nusselt numbers of face 0 (NaN unless it is Dirichlet) */
    double mass_dev, heat_dev;  /* lbm_sums of the final state */
    double t_submit, t_admit, t_done;
    unsigned long long bytes;   /* device footprint */
    long long sites;
    int storage;                /* LBM_STORE_* the request was served in */
} lbm_result;

/* Create a server on the current device with a device-memory budget in bytes (0: 80 % of
 * the free memory) and a residual interval of `chunk` >= 1 steps, queued on `stream`
 * (NULL: a private stream).  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_server_create(unsigned long long budget_bytes, int chunk, void* stream,
                             lbm_server** out);

/* Queue a request: problem p, medium m (NULL: lbm_set_medium defaults), residual tolerance
 * tol > 0 and step limit max_steps >= 1.  Returns its id.  Every lattice lbm_create takes is
 * served: lattices below 512 K sites batch (D3Q15 and node-wall ones too), larger ones step
 * alone; p->scheme ==
 * LBM_SCHEME_AA is kept (one population copy, counted as such against the budget), AUTO is
 * served with two copies.  LBM_EINVAL for an invalid problem, an AA request the scheme does
 * not take (after the storage rule of the serving loop), or one larger than the whole
 * budget. */
lbm_status lbm_server_submit(lbm_server* s, const lbm_params* p, const lbm_medium* m,
                             double tol, long long max_steps, long long* id);

/* One scheduling round: admit what fits, advance every admitted lattice by one chunk, check
 * the residuals, retire finished requests.  Reports the numbers of admitted and queued
 * requests after the round (either pointer may be NULL).  Synchronises. */
lbm_status lbm_server_advance(lbm_server* s, int* n_active, int* n_queued);

/* Give a queued or admitted request host buffers for its final fields: u (3 x ns floats,
 * [3][ns]) and T (ns floats), either may be NULL.  When the request finishes (converged, step
 * limit or unstable) the server writes its macroscopic fields at the final time there, as
 * lbm_macros computes them, before releasing its state.  The buffers are the caller's and must
 * stay valid until the result has been polled.  LBM_EINVAL for an unknown or finished id. */
lbm_status lbm_server_set_output(lbm_server* s, long long id, float* u, float* T);

/* Move up to `max` finished results into out; *n receives how many. */
lbm_status lbm_server_poll(lbm_server* s, lbm_result* out, int max, int* n);

/* Admission policy: LBM_ADMIT_FIFO (the default) or LBM_ADMIT_BACKFILL.  LBM_EINVAL otherwise. */
lbm_status lbm_server_set_policy(lbm_server* s, int policy);

/* Cap the lattice sites admitted at once (0, the default: no cap).  Beyond the sites that
 * fill the GPU, admitting more requests adds no throughput and only delays the earlier
 * ones; with a cap the head of the queue waits until the admitted lattices hold fewer than
 * max_active_sites sites together (a request is always admitted when nothing else is). */
lbm_status lbm_server_set_fill(lbm_server* s, long long max_active_sites);

/* Seconds since lbm_server_create on the server's host clock. */
double lbm_server_clock(const lbm_server* s);

/* Release the server and every request it still holds.  NULL is a no-op. */
void lbm_server_destroy(lbm_server* s);

/* Derived lattice parameters of the context, including the current medium. */
lbm_status lbm_get_lattice(const lbm_ctx* ctx, lbm_lattice* out);

/* Number of time steps taken since create / init. */
long long lbm_steps_done(const lbm_ctx* ctx);

/* Block the host until the context's stream is idle.  Returns LBM_ETIMEOUT (sticky) when a
 * bounded device-side wait of a TMA step ran out since the last check (see LBM_KERNEL_TMA);
 * every other call that synchronises the stream checks the same. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* Text of the last error of the context (never NULL; "" when none).  Owned by ctx. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Static text for a status code. */
const char* lbm_status_string(lbm_status s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_H */
