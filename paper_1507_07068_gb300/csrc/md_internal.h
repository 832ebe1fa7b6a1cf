// md_internal.h -- device data layout and kernel launchers of libmd (sm_103a).
//
// Layout in HBM (all replicas concatenated; "slots" are atom places in cell order):
//   - every replica's slot range starts on a TILE-aligned boundary (tiles never span two
//     replicas, so a CTA's atoms belong to one replica and per-replica sums are plain
//     per-CTA partials); slots past a replica's last atom are padding (never binned,
//     never listed, never integrated);
//   - per-atom SoA arrays: x[3][S], v[3][S], F[3][S], x_build[3][S] (FP64),
//     pos4[S] (int4: position relative to the atom's cell centre in 32-bit fixed point of
//     unit 2^-k A, and the atom's cell coordinates packed in .w; a pair's displacement is
//     an exact integer sum, rounded once when converted to FP32), fm (F'(rho), M'(P) per atom: double2 in FP64
//     mode, float2 in mixed mode), cellc[S] (packed cell coordinates), orig[S] (caller id),
//     fixed[S] (uint8);
//   - Verlet lists in SoA form nbr[k * S + i] (slot of the k-th neighbour of slot i), so a
//     warp reading its 32 atoms' k-th entries reads 128 consecutive bytes, and cnt[S];
//     the Cr-C list the same with indenter slots;
//   - the Cr cell grid: cell_start/cell_count per cell (replica cell ranges concatenated);
//   - the indenter: FP64 SoA positions at t = 0 sorted by their own cell grid (built once),
//     with per-replica displacement z_ind held on the device.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/md.h"

#define MD_TILE 128          // slots per tile; a CTA of the per-atom kernels covers <= one tile
#define MD_RED_CHUNKS 128    // k_reduce: CTAs per replica, each summing a contiguous run of CTA partials
#define MD_ACC 9.6485332e-3  // 1 eV/(A u) in A/fs^2
#define MD_KB 8.617333262e-5 // Boltzmann constant, eV/K
#define MD_CELL_BITS 10      // bits per packed cell coordinate (grids up to 1024 cells per axis)
// Cr-Cr list entry: slot of the neighbour in the low MD_J_BITS bits, and in the top 6 bits
// the direction of its stencil cell: bit 0/1 = x-/x+, 2/3 = y-/y+, 4/5 = z-/z+
#define MD_J_BITS 26
#define MD_J_MASK ((1u << MD_J_BITS) - 1u)

// error bits raised by kernels (device word, read by the host after md_step)
// (MDE_SCHED: a step launched without k_verlet1 found no drift ready - a host bookkeeping error)
// (MDE_LISTCHECK: the debug check after a list build found a violation, see k_check_lists)
enum { MDE_OVERFLOW = 1, MDE_LOST = 2, MDE_SKIN = 4, MDE_COVERFLOW = 8, MDE_SCHED = 16, MDE_LISTCHECK = 32 };
// kinds of violation counted by k_check_lists (DevStatus::chk)
#define MD_NCHK 8
// what k_decide is launched for: an explicit list build (no step), a step whose Task 3 the
// last step's force epilogue made (k_verlet1 runs only if the lists are rebuilt), or a step
// that runs k_verlet1
// DEC_AUTO: k_verlet1 runs when the device's drift flag says no drift is ready or the lists
// are rebuilt (a second graph conditional, set by k_decide)
enum { DEC_BUILD = 0, DEC_DRIFT = 1, DEC_FULL = 2, DEC_AUTO = 3 };
// skin of the inner list (A): rebuilt from the Verlet list when an atom has moved more than
// half of it since the last rebuild
#define MD_INNER_SKIN 0.1

// Hermite cubic coefficients of one table interval, c0 + c1 t + c2 t^2 + c3 t^3
struct alignas(32) Cf64 {
    double x, y, z, w;
};

// FP32 constants of the mixed-precision path, converted once on the host
struct PotF32 {
    float rmin_s_f, inv_hf, rmin_s_m, inv_hm, lf0, beta, f_rc, df_rc, rc;
    float inv_re, d, b0, b1, b2, b3;
    // Eq. A4 in FP32, about t = tc instead of the double root (t = r/r_e - d): with
    // s = (r - rs) / r_e = t - tc, rs = r_e (d + tc) an FP32 number near 0.95 r_e,
    // Phi = t^2 (b0 + b1 s + b2 s^2 + b3 s^3), dPhi/dr = t (c0 + c1 s + c2 s^2 + c3 s^3).
    // About the double root the cubic's terms cancel ~60-fold at the first neighbour shell;
    // about tc (between the first two shells) they do not, and r - rs is exact.
    float c0, c1, c2, c3;
    float tc, rs;
    float D_o, half_ax, inv_yeq, m_rc, dm_rc, rc_m;
    float F_o, n, inv_rho_e, alpha, inv_P_e, rc2;
    int32_t tabulated, nf, nm;
    const float4 *tf, *tp, *tm;
    const float4 *tfp;   // f and Phi coefficients interleaved: [2k] = f, [2k + 1] = Phi
    // direct FP32 forms of the pair loops: f = (re2f / r^2)^ipow when beta = 2 ipow, with
    // re2f = f_e^(1/ipow) r_e^2 (ipow = 0: exp2/log2 form); the shifted-force terms as
    // f(r) - f(rc) - (r - rc) f'(rc) = f(r) - cf - r df_rc, cf = f(rc) - rc f'(rc)
    float re2f, cf;
    int32_t ipow;
};

// potential, passed by value to kernels (lives in the constant bank)
struct PotDev {
    // Eq. A2: f = f_e (r_e/r)^beta = exp2(lf0 - beta log2 r)
    double f_e, r_e, beta, lf0;
    // Eq. A3
    double F_o, n, rho_e, alpha, P_e;
    // Eq. A4 about the double root x = d: with t = r/r_e - d <= 0,
    // Phi = t^2 (b0 + b1 t + b2 t^2 + b3 t^3)   (no cancellation near the cut-off)
    double b[4], d;
    // Eq. A5 with E = exp(-(alpha_x/2)(y/y_eq - 1)): phi = D_o (E^2 - 2E)
    double D_o, half_ax, inv_yeq;
    double rc, rc_m, rc2, rcm2;
    double f_rc, df_rc, m_rc, dm_rc;   // shifted-force constants, 0 when truncating
    int32_t shifted, tabulated;
    // tables: interval k covers [r_min + k h, r_min + (k+1) h]; coefficients c0..c3 of
    // the Hermite cubic in t in [0, 1); forces are d/dr of the same cubic
    double r_min, inv_hf, inv_hm;
    int32_t nf, nm;
    const Cf64 *tf, *tp, *tm;
    const float4 *tf32, *tp32, *tm32;
    PotF32 q;
};

// static per-replica description (read-only on the device)
struct RepDev {
    double lo[3], hi[3], L[3], w[3];  // Cr cell grid; L = hi - lo; w = L / nc (binning)
    double iw[3], iL[3];              // 1 / w, 1 / L (fast path of the exact quotient floors)
    int32_t per[3], nc[3];
    // Fixed-point cell-relative positions (unit u = 2^-k A, DevArgs::qu) are taken about the
    // centres lo + (c + 1/2) wc, wc = Wq u (w rounded to the unit), so two cells' centres
    // differ by an exact multiple Wq of the unit, plus DLq = (L - nc wc) / u (rounded) when
    // a pair crosses a periodic boundary.  w32, dL32: the same in FP32 (prefilters only).
    int32_t Wq[3], DLq[3];
    float w32[3], dL32[3];
    double wc[3];                     // Wq u
    // in the wc frame a cell's box is off by at most c |w - wc| (c < nc): the margin that
    // k_nbr adds to the half-width of a stencil cell's box (with 1e-4 A for FP32 rounding)
    float pad32[3];
    int32_t cell_off, n_cells;           // keys of this replica's cells (n_cells: 8 per 2x2x2 brick)
    int32_t nbk[3];                      // 2x2x2 bricks per axis, ceil(nc / 2)
    int32_t slot_off, n_atoms, n_slots;  // first slot (TILE aligned), real atoms, slots incl. padding
    int32_t real_off;                    // atoms of the replicas before (unpadded)
    int32_t n_mobile;
    // indenter
    int32_t c_off, n_c;                  // indenter slots
    double cg_lo[3], cg_w[3];            // indenter cell grid in its own frame (t = 0)
    int32_t cg_n[3], ccell_off;
    // FP32 copies for the rejection test of k_nbrc: Cr grid origin, box lengths, and the
    // indenter grid's centre and half extent
    float lo32[3], L32[3], iL32[3], cg_ctr32[3], cg_half32[3];
    // dynamics
    double v_ind, dt, mass, acc_per_f;   // acc_per_f = MD_ACC / mass
    double hk;                           // dt acc_per_f / 2, the half-kick factor
    int32_t cen_off[3];                  // per-axis cell centres lo + (c + 1/2) wc in DevArgs::cen
    double z_surface0, zc_min0;
};

// mutable per-replica scalars
struct RepState {
    double z_ind, z_build;               // indenter displacement at the state's time; at the last build
    double z_cur;                        // z_ind at the start of the current step (what a rebuild uses)
    unsigned long long d2b[2];           // max |x - x_build|^2 of the positions in position buffer k
                                         // (bits of a double), for the rebuild test of their time
    int32_t need;                        // rebuild decided for this step
    float dthr, dthr2;                   // mixed: displacements below these (A) cannot decide the rebuild
                                         // test of the positions k_verlet1 / the force epilogue produce
    int32_t rctr;                        // k_reduce: chunks of this replica summed so far (0 between calls)
};

// energies of one replica (device copy of md_energy's sums)
struct RepEnergy {
    double embed, pair, mterm, morse, kinetic, load;
};

// global counters and flags
struct DevStatus {
    int32_t err;            // MDE_* bits
    int32_t any_rebuild;    // rebuild decided this step (host-readable)
    int32_t changed;        // md_set_state: a position or the indenter displacement differs
                            // from the state's (else the forces of the state still hold)
    int32_t max_cnt, max_cntc;
    int32_t pos4_ok;        // pos4 holds every atom's current position about its cell's centre
    int32_t n_cand;         // atoms queued for the Cr-C list search (set by k_nbrc)
    int32_t n_near;         // atoms with Cr-C neighbours (set by k_nbrc_near)
    uint32_t imax_bits;     // mixed: max over atoms of |p - p_in|^2 (FP32 bits) at the positions
                            // this step's k_density uses
    uint32_t imax_next;     // the same for the positions the force epilogue drifted to
    int32_t inner_ok;       // mixed: the inner list is valid for this step's k_density
    int32_t inner_ok_next;  // set by the k_density that rebuilt it; k_decide moves it over
    int32_t drift_ok;       // mixed: the force epilogue already made the next step's Tasks 2-3
    int32_t run_verlet;     // k_verlet1 runs this step (a rebuild, or a step launched as DEC_FULL)
    int32_t imax_fresh;     // the last k_density rebuilt the inner list: every atom's displacement
                            // since is 0 at the positions it used (imax_bits is then stale)
    int64_t step, rebuilds, since_build;
    // position buffers xs[], p4[] in use: the state is in buffer ph & 1 (during a step, from
    // k_decide on, the positions the pair kernels evaluate); the state a step started from
    // is in buffer ph_cur & 1.  k_decide advances ph; md_set_state keeps it.
    int64_t ph, ph_cur;
    unsigned long long chk[MD_NCHK];   // list-check violations by kind (md_check_lists)
};

// everything the kernels need, by value
struct DevArgs {
    int32_t S;               // slots
    int32_t n_rep;
    int32_t total_cells;
    int32_t kmax, kcmax;
    int32_t kinner;          // rows of the inner list: kmax rounded up to a multiple of threads
                             // per atom (its rows are lane-interleaved and padded to the longest
                             // lane's count times the threads per atom)
    int32_t mixed;
    int32_t rebuild_every;
    int32_t debug;               // nonzero: every list build is followed by k_check_lists
    double skin, cut2, cutc2, cut, cutc;
    float qu;                    // unit of the fixed-point positions, 2^-k A
    double qinv;                 // 2^k
    const RepDev *rep;
    RepState *rs;
    RepEnergy *en;
    DevStatus *st;
    const int32_t *tile_rep;     // replica of each tile
    const double *cen;           // cell-centre coordinates per axis (see RepDev::cen_off)
    const int32_t *cell_rep;     // replica of each cell
    // per-atom.  Positions and their FP32 cell-relative copies live in two buffers: during a
    // step, buffer (cur & 1) holds the state the step starts from and buffer (step & 1) the
    // positions the pair kernels use (outside a step both indices name the state).  FP64
    // mode keeps one buffer (both pointers equal).
    double *xs[2];               // [3][S] each
    int4 *p4[2];
    double *v, *F, *xb;          // [3][S]: velocity and force at the state's time, x at the build
    double *vh;                  // [3][S]: v(t + dt/2) of the current step
    double2 *fm64;
    float2 *fm32;
    int32_t *inner, *icnt;       // mixed precision: the inner list, entries of the Verlet list
                                 // within rc + MD_INNER_SKIN when it was last rebuilt
    int4 *pin;                   // mixed: pos4 of each atom when the inner list was rebuilt
    int4 *pb;                    // mixed: pos4 of each atom when the Verlet list was rebuilt
    float rin2, ithr2;           // (rc + MD_INNER_SKIN)^2; max |p - p_in|^2 before a rebuild
    int32_t *cellc, *orig;
    uint8_t *fixed;
    int32_t *nbr, *cnt, *nbrc, *cntc;
    int32_t *cand, *near;        // Cr-C: atoms within reach of an indenter grid / with neighbours
    double *vir;                 // per-atom virial [6][S] (xx yy zz xy xz yz), allocated on first request
    float4 *fmorse;              // mixed precision: Morse force and energy of each atom in near
    // rebuild scratch
    int32_t *key, *perm, *cell_count, *cell_start, *cell_fill, *scan_blk;
    double *sx, *sv, *sF;        // [3][S] gather scratch
    int32_t *sorig;
    uint8_t *sfixed;
    // indenter (sorted by indenter cell)
    const double *xc0;           // [3][C]
    const float4 *xc32;          // [C] position relative to its replica's indenter-grid origin (FP32)
    const int32_t *ccell_start, *ccell_count;
    int32_t C;
    // block partial sums: [6][max_blocks]
    double *part;
    double *rsum;                        // k_reduce scratch: [n_rep][MD_RED_CHUNKS][6] chunk sums
    int32_t max_blocks;
};

// Cell order: 2x2x2 bricks of cells, bricks in row-major order and the eight cells of a
// brick in row-major order, so that a CTA's atoms (~8 cells) fill a compact block whose
// 27-cell stencil covers 64 cells (a row of 8 cells: 90).  Keys of cells past an odd grid's
// last row stay empty.
__host__ __device__ __forceinline__ int cell_key_loc(const RepDev &R, int c0, int c1, int c2)
{
    return ((((c2 >> 1) * R.nbk[1] + (c1 >> 1)) * R.nbk[0] + (c0 >> 1)) << 3) | ((c2 & 1) << 2) |
           ((c1 & 1) << 1) | (c0 & 1);
}
__host__ __device__ __forceinline__ void key_cell_loc(const RepDev &R, int loc, int &c0, int &c1, int &c2)
{
    const int b = loc >> 3, l = loc & 7;
    c0 = 2 * (b % R.nbk[0]) + (l & 1);
    c1 = 2 * ((b / R.nbk[0]) % R.nbk[1]) + ((l >> 1) & 1);
    c2 = 2 * (b / (R.nbk[0] * R.nbk[1])) + (l >> 2);
}

struct LaunchCfg {
    int32_t tpa;            // threads per atom
    int32_t block;          // threads per block
    int32_t max_rep_slots;  // slots of the largest replica (k_reduce's chunks per replica)
};

// ---- host-side helpers implemented in md_kernels.cu
int md_build_pot(const md_params *p, PotDev *out, Cf64 **d_tabs64, float4 **d_tabs32, char *err, size_t errlen);

// ---- launchers (all enqueue on `s`; return cudaError_t of the launch)
cudaError_t launch_decide(const DevArgs &a, int mode, int use_cond, cudaGraphConditionalHandle h, cudaStream_t s,
                          cudaGraphConditionalHandle hv = 0);
cudaError_t launch_rebuild(const DevArgs &a, cudaStream_t s);
cudaError_t launch_verlet1(const DevArgs &a, cudaStream_t s);
// energies = 0: the mixed-precision kernel leaves the embedding-energy partials alone
cudaError_t launch_density(const DevArgs &a, const PotDev &p, const LaunchCfg &c, int energies, cudaStream_t s);
// energies = 0: the mixed-precision force kernel leaves the energy partials alone (k_reduce
// must follow a launch with energies = 1); the FP64 one always writes them
cudaError_t launch_force(const DevArgs &a, const PotDev &p, const LaunchCfg &c, int integrate, int energies,
                         cudaStream_t s);
// the debug check of the lists of the last build: counters DevStatus::chk cleared, then
// every atom's lists checked against `radius` (<= 0: the list radius rc + skin)
cudaError_t launch_check_lists(const DevArgs &a, double radius, cudaStream_t s);
// the Morse sums alone (mixed precision), and the force kernel with or without them first
cudaError_t launch_morse(const DevArgs &a, const PotDev &p, cudaStream_t s);
cudaError_t launch_force_split(const DevArgs &a, const PotDev &p, const LaunchCfg &c, int integrate, int energies,
                               int with_morse, cudaStream_t s);
cudaError_t launch_reduce(const DevArgs &a, const LaunchCfg &c, cudaStream_t s);
// per-atom virial of every atom at the state positions into a.vir (uses the lists and the
// F', M' of the last force evaluation, which are those of the state)
cudaError_t launch_virial(const DevArgs &a, const PotDev &p, const LaunchCfg &c, cudaStream_t s);
// before a force pass with integrate = 2 (mixed precision): thresholds and accumulators of
// the drift it makes
cudaError_t launch_drift_prep(const DevArgs &a, cudaStream_t s);
// md_set_state for replica r (n atoms from slot slot_off): clear the error word, set z_ind
// and the step count, then (stage = new positions in caller order, or NULL to keep them)
// store the positions, their pos4, the exact displacement test against the last build
// (d2b of replica r) and the inner list's displacement test, then any_rebuild by the
// displacement rule over every replica
cudaError_t launch_state_set(const DevArgs &a, int r, int slot_off, int n, double z_ind, long long step,
                             const double *stage, cudaStream_t s);

// ---- allocation-free small-system evaluation (md_forces_small): all pairs, FP64 forms
enum { MD_SMALL_BLOCK = 128, MD_SMALL_MAX_BLOCKS = MD_SMALL_MAX_ATOMS / MD_SMALL_BLOCK };
struct SmallArgs {
    int32_t n, n_c, nb;                  // film atoms, indenter atoms, CTAs
    const double *x, *xc;                // caller's AoS positions (n x 3, n_c x 3)
    double L[3], iL[3];
    int32_t per[3];
    double *F, *energy;                  // caller's outputs
    double *fm;                          // scratch: F'(rho_i), M'(P_i) interleaved (2n)
    double *part;                        // scratch: per-CTA energy sums [4][nb]
};
// analytic FP64 forms of md_params into P (no tables; allocates nothing)
int md_pot_forms(const md_params *p, PotDev *P, char *err, size_t errlen);
// address and length (doubles) of the static scratch on the current device; also loads
// the three kernels of launch_small
cudaError_t small_setup(double **scratch, size_t *n_doubles);
cudaError_t launch_small(const SmallArgs &g, const PotDev &P, cudaStream_t s);
