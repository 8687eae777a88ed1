/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the 3D double-distribution-function
 * MRT lattice Boltzmann model for convection in porous media at the REV scale
 * (Liu & He, arXiv:1611.03329).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the tests, the package's smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order (Sec. 3):
 *   1. gather the pre-collision populations f_i(x,t) = f_i*(x - e_i, t-1),
 *      g_i(x,t) = g_i*(x - e_i, t-1) (streaming, Eqs. 10 and 35) with the wall rules;
 *   2. sigma*T = sum g_i (Eq. 39);
 *   3. G = buoy*(T - T0) + a (Eq. 5);
 *   4. rho = sum f_i (Eq. 25); v, l0, l1 (Eq. 28, sum over ALL i); u (Eq. 27);
 *   5. F (Eq. 4);
 *   6. m = M f with the dense 19x19 matrix typed from Eq. A2 (D3Q15: the 15x15 matrix of
 *      Eq. A1, velocities of Eq. 12, f_eq of Eq. 18, m_eq of Eq. 15, S~ of Eq. 17, Lambda of
 *      Eq. 16);
 *   7. m_eq = M f_eq with f_eq from Eq. 24 (Eq. 11);
 *   8. S~ from Eq. 23;
 *   9. m* = m - Lambda (m - m_eq) + (I - Lambda/2) S~ (Eq. 9, dt = 1);
 *  10. f* = M^-1 m* with M^-1 from a Gauss-Jordan inverse of M;
 *  11. n = N g (Eq. 36); n_eq (Eq. 37); n* = n - Q (n - n_eq) (Eq. 34);
 *      g* = N^-1 n* with N^-1 typed from Eq. 43;
 *  12. store f*, g* in the other array.
 * With the enthalpy model (App. B) step 2 becomes En_e = sum g (Eq. B7) with T and f_l from
 * Eqs. B8-B9, the flow is collided only where f_l >= 0.5 (elsewhere f rests at f_eq(rho, 0)
 * and u = 0; the FP64 value of f_l decides), and step 11 uses n_eq of Eq. B6 with
 * zeta_alpha from Eq. B11.  The oracle records, per site, how close f_l came to the gate
 * (orc_gate_margin), so that a check against a lower-precision implementation can tell the
 * sites where the two may legitimately decide differently.
 *
 * Boundary rules (the paper uses non-equilibrium extrapolation; this oracle follows the
 * halfway rules that the GPU library implements, Eqs. 10 and 35 in pull form):
 *   periodic faces wrap; a no-slip wall gives f_i(x) = f_opp(i)*(x); a moving wall or
 *   velocity inlet gives f_i(x) = f_opp(i)*(x) + 2 w_i rho0 (e_i . u_w) / cs^2; an adiabatic
 *   face gives g_i(x) = g_opp(i)*(x); a Dirichlet face (anti-bounce-back) gives
 *   g_i(x) = -g_opp(i)*(x) + 2 omega_i sigma T_w; the convective outflow on the x-high face
 *   gives p(N-1, t+1) = (p(N-1, t) + U p(N-2, t+1)) / (1 + U) for every pre-collision
 *   population p that enters from outside, after which the populations set by that rule
 *   are shifted by w_i (rho0 - rho) / sum(w_i) so that the outlet density is rho0 (the
 *   pressure anchor).  When a diagonal source lies outside two faces, a no-slip wall wins
 *   over a velocity face, which wins over the outflow.
 *
 * Node walls by non-equilibrium extrapolation (the paper's scheme [50], Sec. 4): on a face of
 * kind BC_NEE the layer of nodes on the face is the wall, moving at face_u, at temperature
 * face_T (HT_NEE_DIRICHLET) or at the temperature of the fluid beside it (HT_NEE_ADIABATIC).
 * A wall node x_b does not stream.  With x_f the fluid node beside it (x_b plus the inward
 * normal of every node-wall face it lies on), Guo's rule builds its populations from the
 * wall's equilibrium and the streamed non-equilibrium part of x_f,
 *   f(x_b) = f_eq(rho_b, u_w) + [f(x_f) - f_eq(rho_f, u_f)],
 *   g(x_b) = g_eq(T_b, u_w) + [g(x_f) - g_eq(T_f, u_f)],
 * and they then collide (Eqs. 9, 34) at the wall node's own state: the velocity prescribed as
 * u_w, F from Eq. 4 at u_w, T = T_b (the sum of g).  rho_b = rho_f, except on a wall that
 * withdraws fluid (u_w along its outward normal), which holds rho0: with rho_b = rho_f at
 * both walls the mean density of a transpiring channel drifts.
 *
 * Layout: every array is x-fastest, site s = x + nx*(y + ny*z); populations are stored
 * q-major, f[i*ns + s].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q19 19
#define Q15 15
#define QMAX 19
#define Q7 7

/* ---- lattice tables ------------------------------------------------------------- */

/* D3Q19 velocities, Eq. 19 (columns i = 0..18). */
static const int E19[3][Q19] = {
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1}};

/* D3Q19 weights, stated under Eq. 24. */
static const double W19[Q19] = {1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
                                1.0 / 18, 1.0 / 18, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
                                1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* D3Q19 transformation matrix, Eq. A2 (rows in the moment order of Eq. 20). */
static const double M19[Q19][Q19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
    {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1}};

/* D3Q15 velocities, Eq. 12 (columns i = 0..14). */
static const int E15[3][Q15] = {{0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
                                {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
                                {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1}};

/* D3Q15 weights, stated under Eq. 18. */
static const double W15[Q15] = {2.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9,
                                1.0 / 9,  1.0 / 9,  1.0 / 72, 1.0 / 72, 1.0 / 72,
                                1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72, 1.0 / 72};

/* D3Q15 transformation matrix, Eq. A1 (rows in the moment order of Eq. 13). */
static const double M15[Q15][Q15] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-2, -1, -1, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1},
    {16, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 1, 1, 1, 1, -1, -1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, -1, 1, 1, -1}};

/* D3Q7 velocities: the first seven columns of Eq. 12. */
static const int E7[3][Q7] = {{0, 1, -1, 0, 0, 0, 0},
                              {0, 0, 0, 1, -1, 0, 0},
                              {0, 0, 0, 0, 0, 1, -1}};

/* D3Q7 transformation matrix, Eq. 36. */
static const double N7[Q7][Q7] = {{1, 1, 1, 1, 1, 1, 1},  {0, 1, -1, 0, 0, 0, 0},
                                  {0, 0, 0, 1, -1, 0, 0}, {0, 0, 0, 0, 0, 1, -1},
                                  {0, 1, 1, 1, 1, 1, 1},  {0, 1, 1, -1, -1, 0, 0},
                                  {0, 1, 1, 0, 0, -1, -1}};

/* Inverse of N as printed, Eq. 43. */
static const double NINV7[Q7][Q7] = {
    {1, 0, 0, 0, -1, 0, 0},
    {0, 0.5, 0, 0, 1.0 / 6, 1.0 / 6, 1.0 / 6},
    {0, -0.5, 0, 0, 1.0 / 6, 1.0 / 6, 1.0 / 6},
    {0, 0, 0.5, 0, 1.0 / 6, -1.0 / 3, 1.0 / 6},
    {0, 0, -0.5, 0, 1.0 / 6, -1.0 / 3, 1.0 / 6},
    {0, 0, 0, 0.5, 1.0 / 6, 1.0 / 6, -1.0 / 3},
    {0, 0, 0, -0.5, 1.0 / 6, 1.0 / 6, -1.0 / 3}};

static const double CS2 = 1.0 / 3.0; /* c_s^2, c = 1 (Sec. 3.1.2) */

/* M^-1, computed once by Gauss-Jordan elimination with partial pivoting. */
static double MINV19[Q19][Q19];
static double MINV15[Q15][Q15];
static int minv_ready = 0;

/* The flow lattice of a run: D3Q19 (Sec. 3.1.2) or D3Q15 (Sec. 3.1.1). */
typedef struct {
    int q;
    const int* e;       /* e[a * q + i] */
    const double* w;
    const double* m;    /* m[k * q + i] */
    const double* minv; /* minv[i * q + k] */
} flow_lattice;
static const flow_lattice D19 = {Q19, &E19[0][0], W19, &M19[0][0], &MINV19[0][0]};
static const flow_lattice D15 = {Q15, &E15[0][0], W15, &M15[0][0], &MINV15[0][0]};

static int opposite_in(const flow_lattice* D, int i) {
    const int q = D->q;
    for (int j = 0; j < q; ++j)
        if (D->e[j] == -D->e[i] && D->e[q + j] == -D->e[q + i] &&
            D->e[2 * q + j] == -D->e[2 * q + i])
            return j;
    return -1;
}

static int opposite7(int i) {
    for (int j = 0; j < Q7; ++j)
        if (E7[0][j] == -E7[0][i] && E7[1][j] == -E7[1][i] && E7[2][j] == -E7[2][i]) return j;
    return -1;
}

static int invert_matrix(int n, const double* a, double* inv) {
    double* w = (double*)malloc(sizeof(double) * n * 2 * n);
    if (!w) return -1;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            w[r * 2 * n + c] = c < n ? a[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(w[r * 2 * n + col]) > fabs(w[piv * 2 * n + col])) piv = r;
        if (w[piv * 2 * n + col] == 0.0) {
            free(w);
            return -2;
        }
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col * 2 * n + c];
                w[col * 2 * n + c] = w[piv * 2 * n + c];
                w[piv * 2 * n + c] = t;
            }
        double d = w[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) w[col * 2 * n + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = w[r * 2 * n + col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r * 2 * n + c] -= fct * w[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) inv[r * n + c] = w[r * 2 * n + n + c];
    free(w);
    return 0;
}

static void ensure_minv(void) {
    if (!minv_ready) {
        invert_matrix(Q19, &M19[0][0], &MINV19[0][0]);
        invert_matrix(Q15, &M15[0][0], &MINV15[0][0]);
        minv_ready = 1;
    }
}

/* Export the tables so tests can pin them against the lattice definitions. */
void orc_tables(double* e19, double* w19, double* m19, double* minv19, double* e7,
                double* n7, double* ninv7) {
    ensure_minv();
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < Q19; ++i) e19[a * Q19 + i] = E19[a][i];
    for (int i = 0; i < Q19; ++i) w19[i] = W19[i];
    memcpy(m19, M19, sizeof(M19));
    memcpy(minv19, MINV19, sizeof(MINV19));
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < Q7; ++i) e7[a * Q7 + i] = E7[a][i];
    memcpy(n7, N7, sizeof(N7));
    memcpy(ninv7, NINV7, sizeof(NINV7));
}

void orc_tables15(double* e15, double* w15, double* m15, double* minv15) {
    ensure_minv();
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < Q15; ++i) e15[a * Q15 + i] = E15[a][i];
    for (int i = 0; i < Q15; ++i) w15[i] = W15[i];
    memcpy(m15, M15, sizeof(M15));
    memcpy(minv15, MINV15, sizeof(MINV15));
}

/* ---- pointwise formulas ---------------------------------------------------------- */

/* Eqs. 18 and 24 (the same form on either lattice): f_i^eq = w_i { rho + rho0 [ e.u/cs^2 +
 * (e.u)^2/(2 phi cs^4) - |u|^2/(2 phi cs^2) ] }. */
static void feq_on(const flow_lattice* D, double rho, const double* u, double phi, double rho0,
                   double* feq) {
    const int q = D->q;
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < q; ++i) {
        double eu = D->e[i] * u[0] + D->e[q + i] * u[1] + D->e[2 * q + i] * u[2];
        feq[i] = D->w[i] * (rho + rho0 * (eu / CS2 + eu * eu / (2.0 * phi * CS2 * CS2) -
                                          usq / (2.0 * phi * CS2)));
    }
}

void orc_feq15(double rho, const double* u, double phi, double rho0, double* feq) {
    feq_on(&D15, rho, u, phi, rho0, feq);
}

/* Eq. 15 with beta1 = 1, beta2 = -5 (stated with Eq. 18); the conserved moments are rho (m0)
 * and rho0 u (m3, m5, m7), the values of M f_eq. */
void orc_meq15_eq15(double rho, const double* u, double phi, double rho0, double* meq) {
    const double b1 = 1.0, b2 = -5.0;
    double ux = u[0], uy = u[1], uz = u[2];
    double usq = ux * ux + uy * uy + uz * uz;
    meq[0] = rho;
    meq[1] = -rho + rho0 * usq / phi;
    meq[2] = b1 * rho + b2 * rho0 * usq / phi;
    meq[3] = rho0 * ux;
    meq[4] = -7.0 / 3.0 * rho0 * ux;
    meq[5] = rho0 * uy;
    meq[6] = -7.0 / 3.0 * rho0 * uy;
    meq[7] = rho0 * uz;
    meq[8] = -7.0 / 3.0 * rho0 * uz;
    meq[9] = rho0 * (2 * ux * ux - uy * uy - uz * uz) / phi;
    meq[10] = rho0 * (uy * uy - uz * uz) / phi;
    meq[11] = rho0 * ux * uy / phi;
    meq[12] = rho0 * uy * uz / phi;
    meq[13] = rho0 * uz * ux / phi;
    meq[14] = 0.0;
}

/* Eq. 17: forcing term in moment space (D3Q15). */
void orc_stilde15(const double* u, const double* F, double phi, double rho0, double* S) {
    double ux = u[0], uy = u[1], uz = u[2], Fx = F[0], Fy = F[1], Fz = F[2];
    double uF = ux * Fx + uy * Fy + uz * Fz;
    S[0] = 0.0;
    S[1] = 2.0 * rho0 * uF / phi;
    S[2] = -10.0 * rho0 * uF / phi;
    S[3] = rho0 * Fx;
    S[4] = -7.0 / 3.0 * rho0 * Fx;
    S[5] = rho0 * Fy;
    S[6] = -7.0 / 3.0 * rho0 * Fy;
    S[7] = rho0 * Fz;
    S[8] = -7.0 / 3.0 * rho0 * Fz;
    S[9] = 2.0 * rho0 * (2 * ux * Fx - uy * Fy - uz * Fz) / phi;
    S[10] = 2.0 * rho0 * (uy * Fy - uz * Fz) / phi;
    S[11] = rho0 * (ux * Fy + uy * Fx) / phi;
    S[12] = rho0 * (uy * Fz + uz * Fy) / phi;
    S[13] = rho0 * (ux * Fz + uz * Fx) / phi;
    S[14] = 0.0;
}

/* Eq. 24 on the D3Q19 lattice. */
void orc_feq19(double rho, const double* u, double phi, double rho0, double* feq) {
    feq_on(&D19, rho, u, phi, rho0, feq);
}

/* Eq. 21 with beta1 = 3, beta2 = -5.5, beta3 = -0.5 (stated under Eq. 23); the conserved
 * moments are rho (m0) and rho0 u (m3, m5, m7), the values of M f_eq. */
void orc_meq19_eq21(double rho, const double* u, double phi, double rho0, double* meq) {
    const double b1 = 3.0, b2 = -5.5, b3 = -0.5;
    double ux = u[0], uy = u[1], uz = u[2];
    double usq = ux * ux + uy * uy + uz * uz;
    meq[0] = rho;
    meq[1] = -11.0 * rho + 19.0 * rho0 * usq / phi;
    meq[2] = b1 * rho + b2 * rho0 * usq / phi;
    meq[3] = rho0 * ux;
    meq[4] = -2.0 / 3.0 * rho0 * ux;
    meq[5] = rho0 * uy;
    meq[6] = -2.0 / 3.0 * rho0 * uy;
    meq[7] = rho0 * uz;
    meq[8] = -2.0 / 3.0 * rho0 * uz;
    meq[9] = rho0 * (2 * ux * ux - uy * uy - uz * uz) / phi;
    meq[10] = b3 * meq[9];
    meq[11] = rho0 * (uy * uy - uz * uz) / phi;
    meq[12] = b3 * meq[11];
    meq[13] = rho0 * ux * uy / phi;
    meq[14] = rho0 * uy * uz / phi;
    meq[15] = rho0 * uz * ux / phi;
    meq[16] = meq[17] = meq[18] = 0.0;
}

/* Eq. 23: forcing term in moment space. */
void orc_stilde19(const double* u, const double* F, double phi, double rho0, double* S) {
    double ux = u[0], uy = u[1], uz = u[2], Fx = F[0], Fy = F[1], Fz = F[2];
    double uF = ux * Fx + uy * Fy + uz * Fz;
    S[0] = 0.0;
    S[1] = 38.0 * rho0 * uF / phi;
    S[2] = -11.0 * rho0 * uF / phi;
    S[3] = rho0 * Fx;
    S[4] = -2.0 / 3.0 * rho0 * Fx;
    S[5] = rho0 * Fy;
    S[6] = -2.0 / 3.0 * rho0 * Fy;
    S[7] = rho0 * Fz;
    S[8] = -2.0 / 3.0 * rho0 * Fz;
    S[9] = 2.0 * rho0 * (2 * ux * Fx - uy * Fy - uz * Fz) / phi;
    S[10] = -rho0 * (2 * ux * Fx - uy * Fy - uz * Fz) / phi;
    S[11] = 2.0 * rho0 * (uy * Fy - uz * Fz) / phi;
    S[12] = -rho0 * (uy * Fy - uz * Fz) / phi;
    S[13] = rho0 * (ux * Fy + uy * Fx) / phi;
    S[14] = rho0 * (uy * Fz + uz * Fy) / phi;
    S[15] = rho0 * (ux * Fz + uz * Fx) / phi;
    S[16] = S[17] = S[18] = 0.0;
}

/* Eq. 42: g_i^eq = omega_i T (sigma + e_i.u / c_sT^2), omega_0 = 1 - varpi,
 * omega_1..6 = varpi/6, c_sT^2 = varpi/3. */
void orc_geq7(double T, const double* u, double sigma, double varpi, double* geq) {
    double csT2 = varpi / 3.0;
    for (int i = 0; i < Q7; ++i) {
        double om = i == 0 ? 1.0 - varpi : varpi / 6.0;
        double eu = E7[0][i] * u[0] + E7[1][i] * u[1] + E7[2][i] * u[2];
        geq[i] = om * T * (sigma + eu / csT2);
    }
}

/* Eq. 37: n_eq = T (sigma, ux, uy, uz, varpi sigma, 0, 0). */
void orc_neq7(double T, const double* u, double sigma, double varpi, double* neq) {
    neq[0] = T * sigma;
    neq[1] = T * u[0];
    neq[2] = T * u[1];
    neq[3] = T * u[2];
    neq[4] = T * varpi * sigma;
    neq[5] = 0.0;
    neq[6] = 0.0;
}

/* Eq. 4: F = -(phi nu / K) u - (phi F_phi / sqrt K) |u| u + phi G. */
void orc_force(const double* u, const double* G, double phi, double nu, double K, double Fphi,
               double* F) {
    double umag = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int a = 0; a < 3; ++a)
        F[a] = -(phi * nu / K) * u[a] - (phi * Fphi / sqrt(K)) * umag * u[a] + phi * G[a];
}

/* Eqs. 27-28: explicit solution of the nonlinear Eq. 26 for u (dt = 1).  The sum in v runs
 * over all velocities of the lattice (the printed upper limit 8 is read as a misprint). */
static void velocity_on(const flow_lattice* D, const double* f, const double* G, double phi,
                        double nu, double K, double Fphi, double rho0, double* u) {
    double v[3];
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int i = 0; i < D->q; ++i) s += D->e[a * D->q + i] * f[i];
        v[a] = s / rho0 + 0.5 * phi * G[a];
    }
    double l0 = 0.5 * (1.0 + phi * 0.5 * nu / K);
    double l1 = phi * 0.5 * Fphi / sqrt(K);
    double vmag = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double den = l0 + sqrt(l0 * l0 + l1 * vmag);
    for (int a = 0; a < 3; ++a) u[a] = v[a] / den;
}

void orc_velocity(const double* f, const double* G, double phi, double nu, double K,
                  double Fphi, double rho0, double* u) {
    velocity_on(&D19, f, G, phi, nu, K, Fphi, rho0, u);
}

void orc_velocity15(const double* f, const double* G, double phi, double nu, double K,
                    double Fphi, double rho0, double* u) {
    velocity_on(&D15, f, G, phi, nu, K, Fphi, rho0, u);
}

/* ---- lattice parameters and state -------------------------------------------------- */

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_VELOCITY = 2, BC_OUTFLOW = 3, BC_NEE = 4 };
enum { HT_PERIODIC = 0, HT_ADIABATIC = 1, HT_DIRICHLET = 2, HT_OUTFLOW = 3, HT_NEE_DIRICHLET = 4,
       HT_NEE_ADIABATIC = 5 };

typedef struct {
    int nx, ny, nz;
    double rho0, T0, sigma, varpi;
    double s[QMAX];        /* Lambda, Eq. 22 (D3Q15: the first 15, Eq. 16) */
    double zeta_T, zeta_e, zeta_nu; /* Q, Eq. 38 (zeta_alpha from alpha_e, Eq. 41) */
    double alpha_f;        /* fluid thermal diffusivity */
    double alpha_m;        /* matrix diffusivity; < 0 selects alpha_e = Gamma * alpha_f */
    double Gamma;
    double nu;             /* fluid kinematic viscosity of Eq. 4 and Eq. 28 */
    double phi, K, F_phi;  /* uniform medium; F_phi < 0 selects Ergun's Eq. 6 */
    double phi_ref;        /* porosity at which a porosity field has permeability K */
    double buoy[3];        /* G = buoy (T - T0) + accel, Eq. 5 */
    double accel[3];
    int flow_bc[6];
    int heat_bc[6];
    double face_T[6];
    double face_u[6][3];
    double U_out;          /* advection speed of the convective outflow */
    /* enthalpy-based D3Q7 model for solid-liquid phase change (App. B) */
    int enthalpy;          /* 1: g carries the effective enthalpy En_e (Eq. B7) */
    int flow_off;          /* 1: u = 0 everywhere (conduction melting) */
    double c_pl, c_ref;    /* liquid and reference specific heats (Eq. B13) */
    double sigma_s, sigma_l; /* heat-capacity ratios of the solid and liquid regions (Eq. B4) */
    double T_s, T_l;       /* solidus and liquidus temperatures */
    double L_a;            /* latent heat */
    double alpha_s, alpha_l; /* diffusivities of the solid and liquid phases */
    int q;                 /* flow lattice: 19 (D3Q19, Sec. 3.1.2) or 15 (D3Q15, Sec. 3.1.1) */
} orc_lattice;

static const flow_lattice* lattice_of(const orc_lattice* L) { return L->q == Q15 ? &D15 : &D19; }

typedef struct {
    orc_lattice L;
    long ns;
    double* f;  /* post-collision populations f*(x, t-1) */
    double* g;
    double* fn; /* scratch for the next step */
    double* gn;
    double* phi_site; /* NULL for a uniform medium */
    /* convective outflow history: pre-collision populations entering at x = nx-1 */
    double* pf; /* [5][ny*nz] */
    double* pg; /* [ny*nz]  */
    double* pfn;
    double* pgn;
    long steps;
    /* enthalpy model: per site, the smallest |f_l - 1/2| met by the flow gate in the steps
     * since the last orc_gate_margin_reset (0.5 for a site that never left a pure phase) */
    double* gate_margin;
} orc_state;

/* Directions that enter the domain across the x-high face (e_x = -1): 2, 8, 10, 12 and 14
 * on both lattices (Eqs. 12 and 19). */
static int outflow_slot(int i) {
    static const int slot[Q19] = {-1, -1, 0, -1, -1, -1, -1, -1, 1, -1,
                                  2,  -1, 3, -1, 4,  -1, -1, -1, -1};
    return slot[i];
}

static inline long site_index(const orc_lattice* L, int x, int y, int z) {
    return (long)x + (long)L->nx * ((long)y + (long)L->ny * z);
}

/* Porosity, permeability and Forchheimer coefficient at a site (Eq. 6 for a field). */
static void medium_at(const orc_state* S, long s, double* phi, double* K, double* Fphi) {
    const orc_lattice* L = &S->L;
    if (S->phi_site) {
        double p = S->phi_site[s];
        double kc = p * p * p / ((1.0 - p) * (1.0 - p));
        double kc_ref = L->phi_ref * L->phi_ref * L->phi_ref /
                        ((1.0 - L->phi_ref) * (1.0 - L->phi_ref));
        *phi = p;
        *K = L->K * kc / kc_ref;
        *Fphi = L->F_phi < 0 ? 1.75 / sqrt(150.0 * p * p * p) : L->F_phi;
    } else {
        *phi = L->phi;
        *K = L->K;
        *Fphi = L->F_phi < 0 ? 1.75 / sqrt(150.0 * L->phi * L->phi * L->phi) : L->F_phi;
    }
}

/* Eq. 41 solved for zeta_alpha with alpha_e = phi alpha_f + (1-phi) alpha_m (Sec. 2), or
 * alpha_e = Gamma alpha_f (Eq. 7) when no matrix diffusivity is given. */
static double zeta_alpha_at(const orc_lattice* L, double phi) {
    double alpha_e = L->alpha_m < 0 ? L->Gamma * L->alpha_f
                                    : phi * L->alpha_f + (1.0 - phi) * L->alpha_m;
    double csT2 = L->varpi / 3.0;
    return 1.0 / (0.5 + alpha_e / (L->sigma * csT2));
}

/* Face crossed when the source coordinate c leaves [0, n) on axis a, or -1. */
static int crossed_face(int a, int c, int n) {
    if (c < 0) return 2 * a;
    if (c >= n) return 2 * a + 1;
    return -1;
}

/* Pull of f_i at (x,y,z) ignoring the outflow rule (used for the outlet's inner neighbour,
 * whose x-source always lies inside). */
static double pull_f(const orc_state* S, const double* fp, int i, int x, int y, int z,
                     int use_outflow, const double* hist, int* via_outflow);

static double pull_f_core(const orc_state* S, const double* fp, int i, int x, int y, int z,
                          int use_outflow, const double* hist, int* via_outflow) {
    const orc_lattice* L = &S->L;
    const flow_lattice* D = lattice_of(L);
    const int q = D->q;
    int n[3] = {L->nx, L->ny, L->nz};
    int c[3] = {x - D->e[i], y - D->e[q + i], z - D->e[2 * q + i]};
    int faces[3] = {-1, -1, -1};
    int any = 0;
    for (int a = 0; a < 3; ++a) {
        int fc = crossed_face(a, c[a], n[a]);
        if (fc >= 0 && L->flow_bc[fc] == BC_PERIODIC) {
            c[a] = (c[a] + n[a]) % n[a];
            fc = -1;
        }
        faces[a] = fc;
        if (fc >= 0) any = 1;
    }
    if (!any) return fp[(long)i * S->ns + site_index(L, c[0], c[1], c[2])];
    long here = site_index(L, x, y, z);
    int io = opposite_in(D, i);
    for (int a = 0; a < 3; ++a)
        if (faces[a] >= 0 && L->flow_bc[faces[a]] == BC_WALL) return fp[(long)io * S->ns + here];
    for (int a = 0; a < 3; ++a)
        if (faces[a] >= 0 && L->flow_bc[faces[a]] == BC_VELOCITY) {
            const double* uw = L->face_u[faces[a]];
            double eu = D->e[i] * uw[0] + D->e[q + i] * uw[1] + D->e[2 * q + i] * uw[2];
            return fp[(long)io * S->ns + here] + 2.0 * D->w[i] * L->rho0 * eu / CS2;
        }
    /* remaining case: the x-high convective outflow */
    if (!use_outflow) return 0.0; /* unreachable for valid configurations */
    if (via_outflow) *via_outflow = 1;
    double inner = pull_f(S, fp, i, x - 1, y, z, 0, hist, NULL);
    double old = hist[(long)outflow_slot(i) * L->ny * L->nz + y + (long)L->ny * z];
    return (old + L->U_out * inner) / (1.0 + L->U_out);
}

static double pull_f(const orc_state* S, const double* fp, int i, int x, int y, int z,
                     int use_outflow, const double* hist, int* via_outflow) {
    return pull_f_core(S, fp, i, x, y, z, use_outflow, hist, via_outflow);
}

static double pull_g(const orc_state* S, const double* gp, int i, int x, int y, int z,
                     int use_outflow, const double* hist) {
    const orc_lattice* L = &S->L;
    int n[3] = {L->nx, L->ny, L->nz};
    int c[3] = {x - E7[0][i], y - E7[1][i], z - E7[2][i]};
    int face = -1;
    for (int a = 0; a < 3; ++a) {
        int fc = crossed_face(a, c[a], n[a]);
        if (fc >= 0 && L->heat_bc[fc] == HT_PERIODIC) {
            c[a] = (c[a] + n[a]) % n[a];
            fc = -1;
        }
        if (fc >= 0) face = fc;
    }
    if (face < 0) return gp[(long)i * S->ns + site_index(L, c[0], c[1], c[2])];
    long here = site_index(L, x, y, z);
    int io = opposite7(i);
    if (L->heat_bc[face] == HT_ADIABATIC) return gp[(long)io * S->ns + here];
    if (L->heat_bc[face] == HT_DIRICHLET) {
        /* twice the even part of the wall equilibrium: omega sigma T_w (Eq. 42) or
         * varpi c_ref T_w / 6 (Eq. B12) */
        double om = L->varpi / 6.0;
        double c = L->enthalpy ? L->c_ref : L->sigma;
        return -gp[(long)io * S->ns + here] + 2.0 * om * c * L->face_T[face];
    }
    /* convective outflow on the x-high face */
    if (!use_outflow) return 0.0;
    double inner = pull_g(S, gp, i, x - 1, y, z, 0, hist);
    double old = hist[y + (long)L->ny * z];
    return (old + L->U_out * inner) / (1.0 + L->U_out);
}

/* ---- enthalpy model (App. B) ---------------------------------------------------------- */

/* Eqs. B8 and B9: temperature and liquid fraction from the effective enthalpy, with
 * En_{e,s} = sigma_s c_pl T_s and En_{e,l} = sigma_l c_pl T_l + phi L_a. */
void orc_enthalpy_state(const orc_lattice* L, double phi, double En, double* T, double* fl) {
    double Es = L->sigma_s * L->c_pl * L->T_s;
    double El = L->sigma_l * L->c_pl * L->T_l + phi * L->L_a;
    if (En <= Es) {
        *T = En / (L->sigma_s * L->c_pl);
        *fl = 0.0;
    } else if (En >= El) {
        *T = L->T_l + (En - El) / (L->sigma_l * L->c_pl);
        *fl = 1.0;
    } else {
        double frac = (En - Es) / (El - Es);
        *T = L->T_s + frac * (L->T_l - L->T_s);
        *fl = frac;
    }
}

/* Effective enthalpy of a phase-pure state at temperature T: solid at or below T_s, else
 * liquid (the inverse of Eq. B8 outside the mushy range). */
double orc_enthalpy_of(const orc_lattice* L, double phi, double T) {
    if (T <= L->T_s) return L->sigma_s * L->c_pl * T;
    return L->sigma_l * L->c_pl * T + phi * L->L_a;
}

/* Eq. B12: g_0 = En - varpi c_ref T, g_i = varpi c_ref T / 6 + (e_i . u) c_pl T / 2. */
void orc_geq7_enthalpy(const orc_lattice* L, double En, double T, const double* u, double* geq) {
    geq[0] = En - L->varpi * L->c_ref * T;
    for (int i = 1; i < Q7; ++i) {
        double eu = E7[0][i] * u[0] + E7[1][i] * u[1] + E7[2][i] * u[2];
        geq[i] = L->varpi * L->c_ref * T / 6.0 + 0.5 * eu * L->c_pl * T;
    }
}

/* ---- one site ------------------------------------------------------------------------ */

/* Collision of one site (steps 2-11 above).  macro = (rho, ux, uy, uz, T). */
static void collide_site(const orc_lattice* L, const double* f, const double* g, double phi,
                         double K, double Fphi, double zeta_alpha, const double* u_wall,
                         double* fout, double* gout, double* macro);

void orc_collide_site(const orc_lattice* L, const double* f, const double* g, double phi,
                      double K, double Fphi, double zeta_alpha, double* fout, double* gout,
                      double* macro) {
    collide_site(L, f, g, phi, K, Fphi, zeta_alpha, NULL, fout, gout, macro);
}

/* The collision above; with u_wall the velocity is prescribed (a node wall) instead of being
 * solved from Eqs. 27-28. */
static void collide_site(const orc_lattice* L, const double* f, const double* g, double phi,
                         double K, double Fphi, double zeta_alpha, const double* u_wall,
                         double* fout, double* gout, double* macro) {
    ensure_minv();
    const flow_lattice* D = lattice_of(L);
    const int q = D->q;
    double sumg = 0.0;
    for (int i = 0; i < Q7; ++i) sumg += g[i];
    double T, fl = 1.0;
    if (L->enthalpy)
        orc_enthalpy_state(L, phi, sumg, &T, &fl); /* Eqs. B7-B9 */
    else
        T = sumg / L->sigma; /* Eq. 39 */
    double G[3];
    for (int a = 0; a < 3; ++a) G[a] = L->buoy[a] * (T - L->T0) + L->accel[a]; /* Eq. 5 */
    double rho = 0.0;
    for (int i = 0; i < q; ++i) rho += f[i]; /* Eq. 25 */
    double u[3];
    if (u_wall)
        for (int a = 0; a < 3; ++a) u[a] = u_wall[a];
    else
        velocity_on(D, f, G, phi, L->nu, K, Fphi, L->rho0, u); /* Eqs. 27-28 */
    double F[3];
    orc_force(u, G, phi, L->nu, K, Fphi, F); /* Eq. 4 */

    double m[QMAX], feq[QMAX], meq[QMAX], S[QMAX], ms[QMAX];
    /* the liquid-fraction gate of the flow (f_l >= 1/2 flows), decided on the FP64 value */
    if (L->enthalpy && (L->flow_off || fl < 0.5)) {
        /* solid (or no flow): the flow is not collided; the populations rest at f_eq(rho, 0) */
        u[0] = u[1] = u[2] = 0.0;
        double zero[3] = {0.0, 0.0, 0.0};
        feq_on(D, rho, zero, phi, L->rho0, fout);
        goto thermal;
    }
    for (int k = 0; k < q; ++k) {
        m[k] = 0.0;
        for (int i = 0; i < q; ++i) m[k] += D->m[k * q + i] * f[i];
    }
    feq_on(D, rho, u, phi, L->rho0, feq);
    for (int k = 0; k < q; ++k) { /* m_eq = M f_eq (Eq. 11) */
        meq[k] = 0.0;
        for (int i = 0; i < q; ++i) meq[k] += D->m[k * q + i] * feq[i];
    }
    if (q == Q15)
        orc_stilde15(u, F, phi, L->rho0, S); /* Eq. 17 */
    else
        orc_stilde19(u, F, phi, L->rho0, S); /* Eq. 23 */
    for (int k = 0; k < q; ++k)
        ms[k] = m[k] - L->s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * L->s[k]) * S[k]; /* Eq. 9 */
    for (int i = 0; i < q; ++i) {
        fout[i] = 0.0;
        for (int k = 0; k < q; ++k) fout[i] += D->minv[i * q + k] * ms[k];
    }

thermal:;
    double n[Q7], neq[Q7], ns[Q7], zeta[Q7];
    zeta[0] = L->zeta_T;
    if (L->enthalpy) /* Eq. B11 with alpha_e = f_l alpha_l + (1 - f_l) alpha_s */
        zeta_alpha = 1.0 / (0.5 + (fl * L->alpha_l + (1.0 - fl) * L->alpha_s) / (L->varpi / 3.0));
    zeta[1] = zeta[2] = zeta[3] = zeta_alpha;
    zeta[4] = L->zeta_e;
    zeta[5] = zeta[6] = L->zeta_nu;
    for (int k = 0; k < Q7; ++k) {
        n[k] = 0.0;
        for (int i = 0; i < Q7; ++i) n[k] += N7[k][i] * g[i];
    }
    if (L->enthalpy) { /* Eq. B6 */
        neq[0] = sumg;
        neq[1] = L->c_pl * T * u[0];
        neq[2] = L->c_pl * T * u[1];
        neq[3] = L->c_pl * T * u[2];
        neq[4] = L->varpi * L->c_ref * T;
        neq[5] = neq[6] = 0.0;
    } else {
        orc_neq7(T, u, L->sigma, L->varpi, neq);
    }
    for (int k = 0; k < Q7; ++k) ns[k] = n[k] - zeta[k] * (n[k] - neq[k]); /* Eq. 34 */
    for (int i = 0; i < Q7; ++i) {
        gout[i] = 0.0;
        for (int k = 0; k < Q7; ++k) gout[i] += NINV7[i][k] * ns[k];
    }
    if (macro) {
        macro[0] = rho;
        macro[1] = u[0];
        macro[2] = u[1];
        macro[3] = u[2];
        macro[4] = T;
    }
}

/* ---- whole lattice ------------------------------------------------------------------ */

static int has_outflow(const orc_lattice* L) { return L->flow_bc[1] == BC_OUTFLOW; }

/* Node-wall faces a site lies on (bit f for face f). */
static int nee_faces(const orc_lattice* L, int x, int y, int z) {
    int c[3] = {x, y, z}, n[3] = {L->nx, L->ny, L->nz}, bits = 0;
    for (int a = 0; a < 3; ++a) {
        if (c[a] == 0 && L->flow_bc[2 * a] == BC_NEE) bits |= 1 << (2 * a);
        if (c[a] == n[a] - 1 && L->flow_bc[2 * a + 1] == BC_NEE) bits |= 1 << (2 * a + 1);
    }
    return bits;
}

static void gather_site(orc_state* S, int x, int y, int z, double* f, double* g, int rec);

/* Post-collision populations of a node-wall site (see the header), and its macroscopic
 * values (rho_b, u_w, T_b). */
static void nee_site(orc_state* S, int x, int y, int z, int bits, double* fo, double* go,
                     double* mac) {
    const orc_lattice* L = &S->L;
    const flow_lattice* D = lattice_of(L);
    int c[3] = {x, y, z};
    int wall = -1, hot = -1;
    for (int f = 0; f < 6; ++f)
        if (bits & (1 << f)) {
            c[f / 2] += (f % 2 == 0) ? 1 : -1;
            if (wall < 0) wall = f;
            if (hot < 0 && L->heat_bc[f] == HT_NEE_DIRICHLET) hot = f;
        }
    /* the fluid node beside the wall: its streamed populations and macroscopic values */
    double f[QMAX], g[Q7], m[5], ftmp[QMAX], gtmp[Q7];
    double phi, K, Fphi, phib, Kb, Fphib;
    gather_site(S, c[0], c[1], c[2], f, g, 0);
    medium_at(S, site_index(L, c[0], c[1], c[2]), &phi, &K, &Fphi);
    orc_collide_site(L, f, g, phi, K, Fphi, zeta_alpha_at(L, phi), ftmp, gtmp, m);
    medium_at(S, site_index(L, x, y, z), &phib, &Kb, &Fphib);
    const double* uw = L->face_u[wall];
    double uf[3] = {m[1], m[2], m[3]};
    double Tb = hot >= 0 ? L->face_T[hot] : m[4];
    /* a wall that withdraws fluid (u_w along its outward normal) holds rho0 */
    double out = wall % 2 == 0 ? -uw[wall / 2] : uw[wall / 2];
    double rhob = out > 0.0 ? L->rho0 : m[0];
    /* Guo's rule: the equilibrium of the wall plus the fluid node's non-equilibrium part */
    double eb[QMAX], ef[QMAX], gb[Q7], gf[Q7];
    feq_on(D, rhob, uw, phib, L->rho0, eb);
    feq_on(D, m[0], uf, phi, L->rho0, ef);
    for (int i = 0; i < D->q; ++i) f[i] += eb[i] - ef[i];
    orc_geq7(Tb, uw, L->sigma, L->varpi, gb);
    orc_geq7(m[4], uf, L->sigma, L->varpi, gf);
    for (int i = 0; i < Q7; ++i) g[i] += gb[i] - gf[i];
    /* then the collision at the wall node's own state, with u = u_w */
    collide_site(L, f, g, phib, Kb, Fphib, zeta_alpha_at(L, phib), uw, fo, go, NULL);
    if (mac) {
        mac[0] = rhob;
        mac[1] = uw[0];
        mac[2] = uw[1];
        mac[3] = uw[2];
        mac[4] = Tb;
    }
}

static void reset_outflow_history(orc_state* S) {
    if (!S->pf) return;
    const orc_lattice* L = &S->L;
    long nyz = (long)L->ny * L->nz;
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y) {
            long s = site_index(L, L->nx - 1, y, z);
            for (int i = 0; i < L->q; ++i) {
                int k = outflow_slot(i);
                if (k >= 0) S->pf[k * nyz + y + (long)L->ny * z] = S->f[(long)i * S->ns + s];
            }
            S->pg[y + (long)L->ny * z] = S->g[2L * S->ns + s];
        }
}

void* orc_create(const orc_lattice* L, const double* phi_field) {
    ensure_minv();
    orc_state* S = (orc_state*)calloc(1, sizeof(orc_state));
    if (!S) return NULL;
    S->L = *L;
    S->ns = (long)L->nx * L->ny * L->nz;
    if (S->L.q != Q15) S->L.q = Q19;
    S->f = (double*)calloc((size_t)S->L.q * S->ns, sizeof(double));
    S->g = (double*)calloc((size_t)Q7 * S->ns, sizeof(double));
    S->fn = (double*)calloc((size_t)S->L.q * S->ns, sizeof(double));
    S->gn = (double*)calloc((size_t)Q7 * S->ns, sizeof(double));
    if (phi_field) {
        S->phi_site = (double*)malloc(sizeof(double) * S->ns);
        memcpy(S->phi_site, phi_field, sizeof(double) * S->ns);
    }
    if (L->enthalpy) {
        S->gate_margin = (double*)malloc(sizeof(double) * S->ns);
        for (long s = 0; s < S->ns; ++s) S->gate_margin[s] = 0.5;
    }
    if (has_outflow(L)) {
        long nyz = (long)L->ny * L->nz;
        S->pf = (double*)calloc(5 * nyz, sizeof(double));
        S->pg = (double*)calloc(nyz, sizeof(double));
        S->pfn = (double*)calloc(5 * nyz, sizeof(double));
        S->pgn = (double*)calloc(nyz, sizeof(double));
    }
    return S;
}

void orc_destroy(void* h) {
    orc_state* S = (orc_state*)h;
    if (!S) return;
    free(S->f);
    free(S->g);
    free(S->fn);
    free(S->gn);
    free(S->phi_site);
    free(S->pf);
    free(S->pg);
    free(S->pfn);
    free(S->pgn);
    free(S->gate_margin);
    free(S);
}

/* Initial state: f = f_eq(rho0, u) and g = g_eq(T, u) at every site, stored as the
 * post-collision populations of step t = 0 (u, T given per site, or uniform if NULL). */
void orc_init_equilibrium(void* h, double T_uniform, const double* T_field, const double* u_field) {
    orc_state* S = (orc_state*)h;
    const orc_lattice* L = &S->L;
    for (long s = 0; s < S->ns; ++s) {
        double phi, K, Fphi;
        medium_at(S, s, &phi, &K, &Fphi);
        double u[3] = {0, 0, 0};
        if (u_field)
            for (int a = 0; a < 3; ++a) u[a] = u_field[a * S->ns + s];
        double T = T_field ? T_field[s] : T_uniform;
        double feq[QMAX], geq[Q7];
        feq_on(lattice_of(L), L->rho0, u, phi, L->rho0, feq);
        if (L->enthalpy)
            orc_geq7_enthalpy(L, orc_enthalpy_of(L, phi, T), T, u, geq);
        else
            orc_geq7(T, u, L->sigma, L->varpi, geq);
        for (int i = 0; i < L->q; ++i) S->f[(long)i * S->ns + s] = feq[i];
        for (int i = 0; i < Q7; ++i) S->g[(long)i * S->ns + s] = geq[i];
    }
    reset_outflow_history(S);
    S->steps = 0;
}

void orc_set_populations(void* h, const double* f, const double* g) {
    orc_state* S = (orc_state*)h;
    memcpy(S->f, f, sizeof(double) * S->L.q * S->ns);
    memcpy(S->g, g, sizeof(double) * Q7 * S->ns);
    reset_outflow_history(S);
}

void orc_get_populations(void* h, double* f, double* g) {
    orc_state* S = (orc_state*)h;
    if (f) memcpy(f, S->f, sizeof(double) * S->L.q * S->ns);
    if (g) memcpy(g, S->g, sizeof(double) * Q7 * S->ns);
}

/* Gather the pre-collision populations of one site; when rec is set, record the outflow
 * history for the next step. */
static void gather_site(orc_state* S, int x, int y, int z, double* f, double* g, int rec) {
    const orc_lattice* L = &S->L;
    const flow_lattice* D = lattice_of(L);
    int outf = has_outflow(L);
    int via[QMAX];
    for (int i = 0; i < D->q; ++i) {
        via[i] = 0;
        f[i] = pull_f(S, S->f, i, x, y, z, outf, S->pf, &via[i]);
    }
    /* Pressure anchor of the outlet: shift the populations that came from the convective
     * rule by w_i * (rho0 - rho) / sum(w_i) so that the outlet density equals rho0. */
    if (outf && x == L->nx - 1) {
        double rho = 0.0, wsum = 0.0;
        for (int i = 0; i < D->q; ++i) {
            rho += f[i];
            if (via[i]) wsum += D->w[i];
        }
        if (wsum > 0.0)
            for (int i = 0; i < D->q; ++i)
                if (via[i]) f[i] += D->w[i] * (L->rho0 - rho) / wsum;
    }
    for (int i = 0; i < Q7; ++i) g[i] = pull_g(S, S->g, i, x, y, z, outf, S->pg);
    if (rec && outf && x == L->nx - 1) {
        long nyz = (long)L->ny * L->nz;
        long yz = y + (long)L->ny * z;
        for (int i = 0; i < D->q; ++i) {
            int k = outflow_slot(i);
            if (k >= 0) S->pfn[k * nyz + yz] = f[i];
        }
        S->pgn[yz] = g[2];
    }
}

void orc_step(void* h, int nsteps) {
    orc_state* S = (orc_state*)h;
    const orc_lattice* L = &S->L;
    for (int t = 0; t < nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < L->nz; ++z) {
            for (int y = 0; y < L->ny; ++y)
                for (int x = 0; x < L->nx; ++x) {
                    long s = site_index(L, x, y, z);
                    double f[QMAX], g[Q7], fo[QMAX], go[Q7];
                    double phi, K, Fphi;
                    int nb = nee_faces(L, x, y, z);
                    if (nb) { /* node wall: extrapolated from the fluid node beside it */
                        nee_site(S, x, y, z, nb, fo, go, NULL);
                        for (int i = 0; i < L->q; ++i) S->fn[(long)i * S->ns + s] = fo[i];
                        for (int i = 0; i < Q7; ++i) S->gn[(long)i * S->ns + s] = go[i];
                        continue;
                    }
                    gather_site(S, x, y, z, f, g, 1);
                    medium_at(S, s, &phi, &K, &Fphi);
                    if (S->gate_margin && !L->flow_off) {
                        /* distance of this step's f_l (Eqs. B7-B9) from the gate at 1/2 */
                        double En = 0.0, T, fl;
                        for (int i = 0; i < Q7; ++i) En += g[i];
                        orc_enthalpy_state(L, phi, En, &T, &fl);
                        double d = fabs(fl - 0.5);
                        if (d < S->gate_margin[s]) S->gate_margin[s] = d;
                    }
                    orc_collide_site(L, f, g, phi, K, Fphi, zeta_alpha_at(L, phi), fo, go, NULL);
                    for (int i = 0; i < L->q; ++i) S->fn[(long)i * S->ns + s] = fo[i];
                    for (int i = 0; i < Q7; ++i) S->gn[(long)i * S->ns + s] = go[i];
                }
        }
        double* tmp;
        tmp = S->f; S->f = S->fn; S->fn = tmp;
        tmp = S->g; S->g = S->gn; S->gn = tmp;
        if (S->pf) {
            tmp = S->pf; S->pf = S->pfn; S->pfn = tmp;
            tmp = S->pg; S->pg = S->pgn; S->pgn = tmp;
        }
        S->steps++;
    }
}

/* Macroscopic fields at the current time (pre-collision state): rho, u (3 x ns), T. */
void orc_macros(void* h, double* rho, double* u, double* T) {
    orc_state* S = (orc_state*)h;
    const orc_lattice* L = &S->L;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L->nz; ++z)
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                long s = site_index(L, x, y, z);
                double f[QMAX], g[Q7], fo[QMAX], go[Q7], mac[5];
                double phi, K, Fphi;
                int nb = nee_faces(L, x, y, z);
                if (nb) {
                    nee_site(S, x, y, z, nb, fo, go, mac);
                } else {
                    gather_site(S, x, y, z, f, g, 0);
                    medium_at(S, s, &phi, &K, &Fphi);
                    orc_collide_site(L, f, g, phi, K, Fphi, zeta_alpha_at(L, phi), fo, go, mac);
                }
                if (rho) rho[s] = mac[0];
                if (u)
                    for (int a = 0; a < 3; ++a) u[a * S->ns + s] = mac[1 + a];
                if (T) T[s] = mac[4];
            }
}

long orc_steps_done(void* h) { return ((orc_state*)h)->steps; }

/* Enthalpy model: copy the per-site gate margins (ns doubles, see orc_state.gate_margin) to
 * out; 0.5 everywhere without the model or with flow_off (no gate). */
void orc_gate_margin(void* h, double* out) {
    orc_state* S = (orc_state*)h;
    for (long s = 0; s < S->ns; ++s) out[s] = S->gate_margin ? S->gate_margin[s] : 0.5;
}

void orc_gate_margin_reset(void* h) {
    orc_state* S = (orc_state*)h;
    if (S->gate_margin)
        for (long s = 0; s < S->ns; ++s) S->gate_margin[s] = 0.5;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_sizeof_lattice(void) { return (int)sizeof(orc_lattice); }
