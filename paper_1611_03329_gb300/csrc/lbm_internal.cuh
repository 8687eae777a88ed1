// Internal declarations shared by the two translation units of the CUDA library
// (kernels and host API).  Not part of the public ABI (include/lbm.h).
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kQ = 19;   // D3Q19 flow populations (Eq. 19)
constexpr int kQT = 7;   // D3Q7 temperature populations (Eq. 12, first seven columns)
constexpr int kOutSlots = 6;  // populations entering across the x-high face: 5 f + 1 g
constexpr int kBlock = 256;   // threads per block of the site kernels
constexpr int kStepMinBlocks = 4;  // resident blocks per SM the step kernel is compiled for
// The 16-bit formats store each D3Q19 deviation f_i - w_i rho0 multiplied by kFlowUnit (a
// power of two, so the scaling is exact): the kernels decode and encode those planes by
// conversion alone and run the flow collision in these units, with the constants that meet
// the populations (KParams frho0, inv_rho0, rho0_10, aqc, bqc) scaled to match.  FP32
// storage uses the unit 1.
constexpr double kFlowUnit = 64.0;

// Everything a site kernel needs, passed by value (__grid_constant__).
struct KParams {
    int nx, ny, nz;
    int nyz;        // ny * nz (outflow history plane)
    int storage;    // 0 FP32, 1 FP16, 2 BF16 (LBM_STORE_*)
    float om0, om1, iom0, iom1;  // D3Q7 weights omega_0, omega_1..6 and their inverses
    int block_threads;  // threads per block of the site kernels (host launch setting)
    long long ns;   // sites
    long long sq;   // elements between consecutive population planes (>= ns, padded)
    int off32;      // every element offset within a population copy fits an int
    int reverse;    // step kernels: sweep the blocks in reverse order (set on alternate steps)

    // boundaries (face bits: 1 << face, faces x-low, x-high, y-low, y-high, z-low, z-high)
    unsigned per_mask;    // periodic faces (flow and heat)
    unsigned wall_mask;   // no-slip walls
    unsigned vel_mask;    // velocity faces
    unsigned nee_mask;    // node walls (non-equilibrium extrapolation)
    float face_dT[6];     // T_w - T0 of fixed-temperature faces
    int heat_kind[6];     // LBM_HEAT_* per face
    float heat_abb[6];    // 2 (varpi/6) sigma (T_w - T0): anti-bounce-back term, deviation form
    float face_u[6][3];   // wall velocity of velocity faces
    float out_a, out_b;   // convective outflow weights 1/(1+U), U/(1+U)

    // fluid and lattice
    float rho0, inv_rho0, sigma, inv_sigma, T0, varpi;
    // the flow populations' unit (kFlowUnit for 16-bit storage, else 1): frho0 = unit * rho0,
    // inv_fu = 1 / unit; inv_rho0 holds 1 / (unit rho0), and rho0_10, aqc, bqc (below) the
    // unit as a factor
    float frho0, inv_fu;
    float s_e, s_eps, s_q, s_nu, s_pi, s_m;        // Lambda (Eq. 22), s_rho = s_j = 1
    float zeta_e, zeta_nu, zeta_alpha;              // Q (Eq. 38), zeta_T = 1
    // collision factors: a = s_k / |M_k|^2, b = (1 - s_k/2) / |M_k|^2 for the rows of Eq. A2
    // (|M_k|^2 = 2394, 252, 40, 36, 72, 12, 24, 4, 8), with 2/3 rho0 folded into the q rows
    float ae, be, aeps, beps, aq, aqc, bqc, anu36, bnu36, api72, hbpi72, anu12, bnu12;
    float api24, hbpi24, anu4, bnu4, am8, rho0_10;
    // D3Q15 (Eq. A1 norms 18, 360, 40, 8; the 12 and 4 rows share anu12 / anu4 above)
    int qf;  // flow populations: 19 (D3Q19) or 15 (D3Q15)
    float ae15, be15, aeps15, beps15, aqc15, bqc15, anu8, bnu8;
    float ze6, zn6;  // zeta_e / 6, zeta_nu / 6 (Eq. 43 columns)
    // enthalpy model (App. B): En_{e,s}, En_{e,l}, 1/(sigma_s c_pl), 1/(sigma_l c_pl),
    // 1/(En_{e,l} - En_{e,s}) (0 when isothermal), phase diffusivities, 3/varpi
    int enthalpy, flow_off;
    float ent_Es, ent_El, ent_is, ent_il, ent_Ts, ent_Tl, ent_idE;
    float c_pl, c_ref, alpha_s, alpha_l, inv_csT2;
    float buoy[3], accel[3];                        // G = buoy (T - T0) + accel (Eq. 5)

    // uniform medium, precomputed (Eqs. 4, 28)
    float phi, inv_phi, l0, l1, c_darcy, c_forch;

    // heterogeneous medium: phi per site, K(phi) = cK phi^3 / (1 - phi)^2 (Eq. 6)
    const float* phi_field;  // device, or nullptr for the uniform medium
    float cK, nu, F_phi;     // F_phi < 0: Ergun per site
    int kinf;                // no Darcy / Forchheimer drag
    int hetero_alpha;        // zeta_alpha per site from alpha_e(phi)
    float alpha_f, alpha_m, inv_sig_csT2;
};

// Population planes of one launch: the 26 planes read (in) and written (out) and the outflow
// history read (hin) and written (hout).
struct Planes {
    const void* in[kQ + kQT];  // element type given by KParams::storage
    void* out[kQ + kQT];
    const float* hin;
    float* hout;
    const float* tin;  // T - T0 per site (16-bit formats only): planes in / out
    float* tout;
    // The same planes as element offsets from one base per side (the planes of a copy are one
    // allocation): plane q of the planes read starts at base_in + off_in[q] elements.  Used by
    // the kernels instantiated with 32-bit offsets, when KParams::off32 is set.
    const void* base_in;
    void* base_out;
    int off_in[kQ + kQT];
    int off_out[kQ + kQT];
};

// One lattice of a batched launch: its parameters, its launch planes for either parity, the
// copy that holds its state when the launch sequence starts, and its part of the flat block
// list (blocks [block_begin, block_begin + gx * gy * ceil(nz / rows)), bx threads along x
// per block, `rows` z-planes per block).
struct BatchLattice {
    KParams p;
    Planes pl[2];
    int cur;
    int block_begin;
    int gx, gy;
    int bx;
    int pad_;
};

// Launch wrappers (defined in lbm_kernels.cu).  All are asynchronous on `st`.
// One time step; `pdl`: launched as a programmatic dependent launch (the kernel may be
// scheduled while the stream's previous kernel drains, and waits for it before loading).
cudaError_t launch_step(const KParams& p, bool outflow, const Planes& pl, bool pdl,
                        cudaStream_t st);
// One time step with two x-adjacent sites per thread (step_pair_kernel): D3Q19, no node
// walls, no enthalpy model, nx even, 32-bit plane offsets (KParams::off32).
cudaError_t launch_step_pair(const KParams& p, bool outflow, const Planes& pl, bool pdl,
                             cudaStream_t st);
// AA pattern (FP32, D3Q19, no outflow; one copy).  Pull step (local = false): pl.in is the
// permuted table of the copy (logical plane q at physical opp(q)), pl.out the identity table.
// Local step (local = true): pl = (in: identity, out: permuted), pw.in = the permuted table.
cudaError_t launch_aa_step(const KParams& p, bool local, const Planes& pl, const Planes& pw,
                           bool pdl, cudaStream_t st);
// The streamed layout left by a pull step back to the swapped layout (pl.out: identity table).
cudaError_t launch_aa_normalize(const KParams& p, const Planes& pl, cudaStream_t st);
cudaError_t launch_macros(const KParams& p, bool outflow, const Planes& pl, float* rho, float* u,
                          float* T, cudaStream_t st);
// Equilibrium state written into pl.out.
cudaError_t launch_init_eq(const KParams& p, const Planes& pl, const double* T_field,
                           const double* u_field, double T_uniform, cudaStream_t st);
// One plane between FP64 full values and the storage format: stored = (v - offset) / scale.
cudaError_t launch_plane_to_dev(int storage, const double* src, void* dst, double offset,
                                double scale, long long n, cudaStream_t st);
cudaError_t launch_plane_to_host(int storage, const void* src, double* dst, double offset,
                                 double scale, long long n, cudaStream_t st);
// D3Q7 planes of a 16-bit format (with its temperature plane) from / to 7 x ns FP64 full
// values in device memory.
cudaError_t launch_g_to_dev(const KParams& p, const Planes& pl, const double* src, cudaStream_t st);
cudaError_t launch_g_to_host(const KParams& p, const Planes& pl, double* dst, cudaStream_t st);
// Outflow history from the planes pl.in.
cudaError_t launch_hist_reset(const KParams& p, const Planes& pl, float* hist, cudaStream_t st);
// FP64 totals of the deviations in pl.in: out[0] = sum f', out[1] = sum g'.
cudaError_t launch_sums(const KParams& p, const Planes& pl, double* partials, int nparts,
                        double* out, cudaStream_t st);
// Nusselt profile and its mean / centre value: out[0] = Nu_3D, out[1] = Nu_mp.
cudaError_t launch_nusselt(const KParams& p, bool outflow, const Planes& pl, int face, double Tw,
                           double scale, double* profile, double* out, cudaStream_t st);
// Residual sums: out = (sum |du|^2, sum |u|^2, sum dT^2, sum T^2, nonfinite count).
cudaError_t launch_residual(const float* u, const float* T, const float* up, const float* Tp,
                            long long ns, double* partials, int nparts, double* out,
                            cudaStream_t st);

// TMA step kernel (lbm_tma.cu).  A copy's 26 population planes form one 4D tensor (x, y, z,
// plane) and its FP32 temperature plane (16-bit formats) a 3D one; each has a map with boxes
// 64 x 4 (x, y) and one with boxes 72 x 4 for the x-shifted planes.  Requires nx % 64 == 0,
// ny >= 4, the D3Q19 lattice, no node walls and no enthalpy model.
constexpr int kTmaTileX = 64, kTmaTileY = 4;
struct TmaMaps {
    CUtensorMap pop64, pop72, t64, t72;
};
struct TmaGrid {
    int tiles_x, tiles_y, ntiles;
    int extra_tx;  // bytes a stage waits for beyond its loads (0; > 0 only to test timeouts)
};
// Sets the kernel's shared-memory limit and returns its persistent grid (blocks) and its
// dynamic shared memory per block.
cudaError_t tma_prepare(const KParams& p, bool outflow, int* blocks, int* smem_bytes);
// One time step reading the copy that `m` and pl.in describe; *err is set to 1 when a staged
// load does not arrive within one second (the blocks then stop early).  extra_tx: see TmaGrid.
cudaError_t launch_step_tma(const KParams& p, bool outflow, const Planes& pl, const TmaMaps& m,
                            int blocks, int extra_tx, int* err, bool pdl, cudaStream_t st);

int reduction_blocks();
// Blocks of the residual reduction over ns sites: reduction_blocks(), or fewer for a small
// lattice (at least 2,048 sites per block), so that its launch takes a few blocks, not 608.
int residual_blocks(long long ns);
// The bounds-checked build's record (-DLBM_BOUNDS_CHECK): *checked = 1 and *first_bad = the
// first out-of-range site index a kernel of lbm_kernels.cu met (-1: none); *checked = 0 in the
// ordinary build.
cudaError_t bounds_report(long long* first_bad, int* checked);
// Physical plane of logical D3Q19 + D3Q7 plane q in the AA scheme's swapped layout: the plane
// of the opposite velocity.
int aa_swapped_plane(int q);
// One time step of every lattice of a batch group (same storage, medium kind, outflow, flow
// lattice qf (19 or 15) and node walls): lattice l reads its planes pl[cur ^ flip]; blk_lat
// maps each of the nblocks blocks to its lattice.  pair: two x-adjacent sites per thread (the
// group's layout counts nx / 2 per row).
cudaError_t launch_batch_step(const BatchLattice* tab, const unsigned short* blk_lat, int nblocks,
                              int block_threads, int rows, int storage, bool het, bool outflow,
                              bool enthalpy, bool off32, bool pair, int qf, bool nee, int flip,
                              cudaStream_t st);
// One time step of the AA lattices of a batch group (FP32, D3Q19, no outflow): lattice l runs a
// pull step when (cur ^ flip) is 0, else a local step; cur holds its AA phase.
cudaError_t launch_batch_aa(const BatchLattice* tab, const unsigned short* blk_lat, int nblocks,
                            int block_threads, int rows, bool het, int flip, cudaStream_t st);
// One lattice of a batched residual: its parameters and the planes of its current copy, the
// macroscopic fields written now (cu: u as 3 x ns, cT) and those of the previous residual (pu,
// pT; nullptr on the first one, when the new fields are compared with themselves), its
// partial sums (5 per block, residual_blocks(ns) blocks) and its 5 totals (device).
struct ResLattice {
    KParams p;
    Planes pl;
    float* cu;
    float* cT;
    const float* pu;
    const float* pT;
    double* partials;
    double* out;
    int nr;
    int pad_;
};
// Residual sums of the n lattices of tab, all with the same medium kind (het), outflow,
// storage and thermal model (enthalpy): for each, the macroscopic fields (as launch_macros
// computes them) and the sums of launch_residual over residual_blocks(ns) blocks, bit for
// bit.  blk maps each of the nblocks blocks to (lattice in tab, block within the lattice).
cudaError_t launch_batch_residual(const ResLattice* tab, const int2* blk, int nblocks, bool het,
                                  bool outflow, int storage, bool enthalpy, cudaStream_t st);
// The totals of the n lattices of tab from their partial sums (finalize of launch_residual).
cudaError_t launch_batch_residual_finish(const ResLattice* tab, int n, cudaStream_t st);
// x-extent of a site-kernel block for a lattice of width nx within block_threads threads.
int block_x(int nx, int block_threads);  // number of partial sums the reductions write (<= partials size)

}  // namespace lbm
