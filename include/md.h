/*
 * md.h -- C ABI of libmd: the per-timestep short-range force evaluation of a Cr film
 * indented by a rigid carbon hemisphere (Pal, Agarwala, Raha & Bhattacharya,
 * arXiv:1507.07068), on one NVIDIA GB300 (sm_103a).
 *
 * One call of md_step advances every replica by whole time steps in the order of the
 * paper's time loop (Fig. 5, Table 1):
 *   Task 1  neighbour-list check and rebuild (Sec. 2.6: rebuild when an atom has moved
 *           more than half the skin; cell binning + Verlet list),
 *   Task 2  rigid indenter moved at constant velocity (Sec. 2.1, 2.5),
 *   Task 3  velocity-Verlet half kick and drift (Appendix Eqs. A11-A12),
 *   Task 4  electron densities, embedding derivatives, EAM + Morse forces and energies
 *           (Eq. (1), Appendix Eqs. A1-A10, A13),
 *   Task 5  closing half kick.
 *
 * Conventions for every function below:
 *   - Units: Angstrom, eV, fs, atomic mass units (u).  Accelerations use
 *     1 eV/(A u) = 9.6485332e-3 A/fs^2.
 *   - Arrays of vectors are AoS x0,y0,z0,x1,... in the caller's own atom order; the
 *     library keeps atoms in its own cell order internally and never exposes it.
 *   - Host pointers are read during the call only (md_init copies everything); output
 *     buffers are caller-owned and must hold the stated number of elements.
 *   - Every function returns MD_OK (0) or an MD_ERR_* code; md_last_error() gives a
 *     one-line description.  No C++ exception crosses this interface.
 *   - A handle is used from one host thread at a time.  All device work runs on the
 *     CUDA stream given to md_init; getters synchronise that stream.
 *   - The library owns all device memory it allocates (cudaMalloc at md_init, freed by
 *     md_free); no allocation happens in md_step.
 */
#ifndef MD_H
#define MD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
    MD_OK = 0,
    MD_ERR_ARG = 1,             /* invalid argument (sizes, box too small for the cell grid, ...) */
    MD_ERR_CUDA = 2,            /* a CUDA runtime call failed; the handle should be freed */
    MD_ERR_NBR_OVERFLOW = 3,    /* an atom had more neighbours than kmax / kcmax at a rebuild */
    MD_ERR_SKIN_VIOLATION = 4,  /* fixed rebuild interval: an atom moved more than skin/2 */
    MD_ERR_LOST_ATOM = 5,       /* an atom left the cell-grid domain along a non-periodic axis (or became NaN) */
    MD_ERR_STATE = 6            /* call not valid in the handle's current state */
};

/* arithmetic of the force kernels */
enum {
    MD_FP64 = 0,    /* everything in FP64 */
    MD_MIXED = 1    /* pair and EAM arithmetic in FP32 on cell-relative positions; FP64
                       integration, skin test, list build and energy/load reductions */
};

/*
 * Potential parameters (Appendix Eqs. A2-A5).  The paper prints the forms but not the
 * values (they come from its refs. [42] and [34]); any consistent set may be passed.
 *   f(r)   = f_e (r_e / r)^beta                                   Eq. A2
 *   F(rho) = -F_o [1 - n ln(rho/rho_e)] (rho/rho_e)^n              Eq. A3 (ln(.)^n read as n ln(.))
 *   M(P)   = alpha u^2 exp(-u^2),  u = P/P_e - 1                   Eq. A3
 *   Phi(x) = (x - d)^2 (a3 x^3 + a2 x^2 + a1 x + a0), x = r/r_e <= d; 0 beyond   Eq. A4
 *   phi(y) = D_o [exp(-alpha_x (y/y_eq - 1)) - 2 exp(-(alpha_x/2)(y/y_eq - 1))] Eq. A5
 * f, f^2 and Phi are cut at rc, phi at rc_morse.  shifted = 1 replaces f and phi below
 * their cut-offs by the shifted-force forms g(r) - g(rc) - (r - rc) g'(rc) (continuous
 * forces; needed for energy conservation); shifted = 0 truncates.  tabulated = 1
 * evaluates f, Phi and phi from cubic Hermite tables on a uniform grid from r_min to the
 * cut-off with spacing <= h (knot values and slopes from the forms above, forces the
 * exact derivative of the interpolant); tabulated = 0 evaluates the forms directly.
 */
typedef struct md_params {
    double r_e, f_e, beta;
    double F_o, n, rho_e;
    double alpha, P_e;
    double a[4];                /* a0, a1, a2, a3 */
    double d;
    double D_o, alpha_x, y_eq;
    double rc, rc_morse;
    int32_t shifted, tabulated;
    double r_min, h;
} md_params;

/*
 * One independent indentation system (a "replica").
 *   x_cr, v_cr : 3*n_cr doubles, film positions (A) and velocities (A/fs)
 *   fixed      : n_cr bytes, nonzero = atom held fixed (v = 0, never moved, still exerts
 *                and feels forces), or NULL for none
 *   x_c        : 3*n_c doubles, indenter atom positions at zero displacement (rigid; at
 *                time t they are x_c + (0, 0, z_indenter(t)), with z_indenter(0) =
 *                z_indenter0); NULL when n_c = 0
 *   box_lo/hi  : the cell-grid domain.  A periodic axis has period hi - lo (minimum image);
 *                along a non-periodic axis an atom outside [lo, hi] is reported as lost.
 *   z_indenter0, v_indenter : indenter displacement at t = 0 and its rate (A/fs; negative
 *                moves the indenter down into the film)
 *   dt (fs), mass_cr (u)
 */
typedef struct md_system {
    int32_t n_cr, n_c;
    const double *x_cr, *v_cr, *x_c;
    const uint8_t *fixed;
    double box_lo[3], box_hi[3];
    int32_t periodic[3];
    double z_indenter0, v_indenter, dt, mass_cr;
} md_system;

/*
 * Options shared by all replicas of a handle.
 *   pot           : potential parameters (copied)
 *   precision     : MD_FP64 or MD_MIXED
 *   skin          : Verlet skin (A); lists hold pairs within rc + skin (Cr-Cr) and
 *                   rc_morse + skin (Cr-C)
 *   rebuild_every : 0 = rebuild when max displacement since the last build exceeds skin/2
 *                   (or, with an indenter, when that plus the indenter's travel exceeds the
 *                   skin); k > 0 = rebuild every k steps (a larger displacement is then
 *                   reported as MD_ERR_SKIN_VIOLATION)
 *   kmax, kcmax   : neighbour capacity per atom for Cr-Cr and Cr-C (0 = defaults 80, 160)
 *   tpa           : threads per atom in the force kernels, 1, 2, 4 or 8 (0 = the smallest
 *                   that puts at least 65 536 threads on all replicas' atoms)
 *   block         : threads per block in the force kernels (0 = default)
 *   use_graph     : nonzero = md_step replays a captured CUDA graph
 *   inner_skin    : MD_MIXED only.  The inner list (Sec. 2.6: the Verlet-list entries the
 *                   density and force loops visit) holds the pairs within rc + inner_skin
 *                   and is rebuilt from the Verlet list when an atom has moved more than
 *                   inner_skin / 2 since its last build; 0 = default 0.1 A; < 0 = rebuilt
 *                   every step with radius rc, as in the paper.  Forces do not depend on
 *                   it: both loops take exactly the pairs within rc, in Verlet-list order.
 *   debug_checks  : nonzero = every list build (in md_step too) is followed by the checks
 *                   of md_check_lists at the list radius; a violation ends the call with
 *                   MD_ERR_STATE and the counts in md_last_error (a debug mode: the check
 *                   costs about as much as the build)
 */
typedef struct md_options {
    const md_params *pot;
    int32_t precision;
    double skin;
    int32_t rebuild_every;
    int32_t kmax, kcmax;
    int32_t tpa, block;
    int32_t use_graph;
    double inner_skin;
    int32_t debug_checks;
} md_options;

/* Energies of one replica after the last force evaluation (eV); FP64 sums. */
typedef struct md_energy {
    double embed;       /* sum_i F(rho_i)                    (Eq. A1)            */
    double pair;        /* 1/2 sum_{i != j} Phi(r_ij)        (Eq. A1)            */
    double mterm;       /* sum_i M(P_i)                      (Eq. A1)            */
    double morse;       /* sum_{i in Cr, c in C} phi(y_ic)   (Eq. A5)            */
    double kinetic;     /* sum_i m v_i^2 / 2                                     */
    double potential;   /* embed + pair + mterm + morse                          */
    double total;       /* potential + kinetic                                   */
    double temperature; /* 2 kinetic / (3 k_B N_mobile)                          */
    double load;        /* z force on the indenter = -sum_i F^Morse_{i,z} (eV/A) */
    double depth;       /* top Cr plane at t = 0 minus the indenter's lowest atom (A) */
    double z_indenter;  /* current indenter displacement (A)                     */
    int64_t step;       /* steps taken                                           */
    int64_t rebuilds;   /* neighbour-list rebuilds after md_init                 */
} md_energy;

/* Per-phase device time of md_step_profiled, milliseconds summed over its steps:
 * skin = the Task 1 decision (with Task 2), rebuild = binning + lists (when decided),
 * verlet1 = Task 3 with the displacement test the next decision uses, density / force =
 * Task 4 (force includes Task 5), morse = the Cr-C sums of the atoms under the indenter
 * (mixed precision: their own kernel, run between density and force here and beside the
 * density kernel in md_step; FP64: inside force, morse = 0).  In mixed precision the
 * force kernel also makes the next step's Task 3 from the state it has just completed
 * (as do the force evaluations of md_init, md_set_state and md_compute_forces); verlet1
 * then runs only on steps that rebuild the lists or follow md_build_neighbors.  reduce =
 * the energy sums, which run once at the end of the call. */
typedef struct md_phase_times {
    double skin, rebuild, verlet1, density, morse, force, reduce;
    int64_t steps, rebuilds;
} md_phase_times;

typedef struct md_handle md_t;

/*
 * Copy n_replicas systems to the device, bin the indenter, build the potential tables,
 * build the neighbour lists and evaluate forces and energies at t = 0 (the accelerations
 * Task 3 needs at the first step).  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream).  On success *out receives a handle to be released with md_free.
 * Errors: MD_ERR_ARG (bad sizes or options, a periodic axis shorter than 3 cells of
 * rc + skin, or an indenter wider than the periodic box allows), MD_ERR_CUDA,
 * MD_ERR_NBR_OVERFLOW.  On error *out is set to NULL and nothing is leaked.
 */
int md_init(const md_system *sys, int32_t n_replicas, const md_options *opt, void *cuda_stream, md_t **out);

/* Task 1 now: wrap positions into periodic boxes, bin all atoms into cells (counting
 * sort of cell keys, ascending caller id within a cell) and rebuild both Verlet lists
 * (Sec. 2.6).  Errors: MD_ERR_NBR_OVERFLOW, MD_ERR_LOST_ATOM, MD_ERR_CUDA. */
int md_build_neighbors(md_t *h);

/* Task 4 at the current positions without integrating: densities, F'(rho), M'(P),
 * forces, energies and load (Eq. (1), Eqs. A1-A10).  Uses the current lists. */
int md_compute_forces(md_t *h);

/* Advance every replica by n >= 0 time steps (Fig. 5: Tasks 1-5 per step).
 * A neighbour list that overflows its capacity (kmax / kcmax) at a rebuild inside the call
 * is recovered: the library grows the capacity past the count it met, returns every
 * replica to the state the call started from, rebuilds the lists there and runs the n
 * steps again (the rebuild count then includes that extra build, and the sums over pairs
 * follow the new lists' order).  For this it keeps a device copy of positions, velocities
 * and indenter state when n >= 16 or when the longest list of the last build came within
 * 1/8 of its capacity (8 entries at least); a call without that copy, and the other device-side errors (lost atom, skin
 * violation), return the error when the call ends, and the state is then not meaningful. */
int md_step(md_t *h, int64_t n);

/* As md_step, launching every kernel directly with CUDA events around each phase, and
 * returning the summed device time per phase in *out (for measurement). */
int md_step_profiled(md_t *h, int64_t n, md_phase_times *out);

/* Energies of replica `replica` (0-based). */
int md_get_energy(md_t *h, int32_t replica, md_energy *out);

/* Forces (eV/A) of the last force evaluation, 3*n_cr doubles in caller order. */
int md_get_forces(md_t *h, int32_t replica, double *out3n);

/* Indenter load (eV/A, positive when the film pushes the indenter up) and depth (A). */
int md_get_indenter_load(md_t *h, int32_t replica, double *load_z, double *depth);

/* Positions (3*n_cr), velocities (3*n_cr) at the current integer time, indenter
 * displacement and step count; any pointer may be NULL. */
int md_get_state(md_t *h, int32_t replica, double *x3n, double *v3n, double *z_ind, int64_t *step);

/* Replace positions and velocities (caller order; x3n or v3n may be NULL to keep), the
 * indenter displacement and the step count of one replica, then re-evaluate forces at the
 * new state -- unless every position and the indenter displacement are bit for bit those
 * already held, when the forces held stay valid (forces do not depend on velocities), and,
 * in mixed precision with the velocities bit for bit those held too, so does the next
 * step's Task 3 that the last force evaluation made (the device checks the velocities as
 * they arrive; the next step reads the result) --
 * (the energy sums of the new state are evaluated when md_get_energy first asks
 * for them; an md_step in between makes its own).  The neighbour lists are kept when the new positions pass the rebuild test of
 * md_step (max |x - x_build| and the indenter's travel since the last build against the
 * skin, Sec. 2.6), else rebuilt (as md_build_neighbors).  The call returns once x3n and v3n
 * have been read (the caller may reuse them).  Errors: MD_ERR_LOST_ATOM,
 * MD_ERR_NBR_OVERFLOW, MD_ERR_CUDA. */
int md_set_state(md_t *h, int32_t replica, const double *x3n, const double *v3n, double z_ind, int64_t step);

/* One exchange of a replica's state with the host around n >= 1 time steps (Fig. 5's time
 * loop driven from outside, e.g. by a serving layer that holds the state between calls):
 * md_set_state(replica, x3n, v3n, z_ind, step), md_step(n), then the replica's positions
 * and velocities into x_out, v_out (3*n_cr doubles each, caller order; they may be x3n and
 * v3n) and its energies into *e_out -- the results of those calls made in turn (the same
 * values bit for bit).  The positions after the last step's Task 3 go back to the host
 * while its density and force passes run (one synchronisation at the end).  Host arrays
 * in page-locked memory copy fastest; all pointers are required.  A list overflow inside
 * the steps is recovered as md_step recovers it (the same checkpoint policy; the redo runs
 * as md_step); handles without graphs make the calls in turn.  Errors: those of
 * md_set_state and md_step; MD_ERR_ARG for a NULL pointer or n < 1. */
int md_step_io(md_t *h, int32_t replica, const double *x3n, const double *v3n, double z_ind, int64_t step,
               int64_t n, double *x_out, double *v_out, md_energy *e_out);

/* Per-atom virial of one replica at the current state, 6 doubles per atom in caller order
 * (xx, yy, zz, xy, xz, yz; eV): the potential part of the per-atom stress times volume
 * (Task 4 can give stresses, Sec. 2.1; their histories are derived along a run, Sec. 3.1).
 * Every pair term of the energy depends on one distance r; with c = (dE/dr)/r the force on
 * i from j is c (x_j - x_i), and each atom of the pair holds half of
 * c (x_j - x_i) (x) (x_j - x_i); a Cr-C pair gives its half to the Cr atom.  The sum over
 * the atoms is the derivative of the energy under a homogeneous deformation.  The kinetic
 * part, -m v (x) v, follows from md_get_state.  The call evaluates the forces again (same
 * values) and then the virial.  Errors: MD_ERR_ARG, MD_ERR_CUDA. */
int md_get_virial(md_t *h, int32_t replica, double *out6n);

/* The indenter's velocity v_ind (A/fs along z; negative = downwards) of one replica from
 * the next step on (Task 2, Sec. 2.1; the loading and unloading legs of an indentation run,
 * Sec. 2.5).  Positions, forces and lists are unchanged; the next step re-derives its
 * displacement test for the new indenter path.  Errors: MD_ERR_ARG, MD_ERR_CUDA. */
int md_set_indenter_velocity(md_t *h, int32_t replica, double v_ind);

/* Test hook (no counterpart in the paper: it exposes the Verlet lists of Sec. 2.6 so that
 * they can be compared set for set with an independent build).  which = 0: Cr-Cr list,
 * which = 1: Cr-C list, as built at the last rebuild.
 * cell_xyz (3*n_cr, may be NULL): cell coordinates of each atom in the Cr cell grid;
 * cnt (n_cr): list lengths (capped at the capacity); nbr (n_cr*kmax, may be NULL): entries
 * in caller ids (film ids for which = 0, indenter ids for which = 1), row i holding atom
 * i's first min(cnt[i], kmax) entries in unspecified order. */
int md_get_neighbors(md_t *h, int32_t replica, int32_t which, int32_t *cell_xyz, int32_t *cnt,
                     int32_t *nbr, int32_t kmax);

/* Debug check of the neighbour lists of the last build (no counterpart in the paper; it
 * stands in for a memory checker by testing, on the device, every invariant the pair
 * kernels rely on when they index memory with list entries).  radius <= 0 means the list
 * radius rc + skin.  out8 (caller-owned, 8 counts over all replicas):
 *   [0] entries outside the atom's replica or naming the atom itself, [1] lengths above the
 *   capacity, [2] direction codes that do not match the two atoms' cells, [3] listed pairs
 *   at or beyond `radius` at the build positions (exact FP64), [4] pairs within `radius`
 *   there that are missing, [5] pairs listed one way only, [6] Cr-C entries outside the
 *   replica's indenter or beyond rc_morse + skin, [7] inner-list entries (MD_MIXED) that are
 *   not in the Verlet list.
 * All zero for lists as built.  With radius < rc + skin, [3] counts the listed pairs between
 * radius and the list radius.  Synchronises the stream.  Errors: MD_ERR_ARG, MD_ERR_CUDA. */
int md_check_lists(md_t *h, double radius, int64_t *out8);

/* Utility (no counterpart in the paper): sizes of one handle.  out[0] = replicas,
 * out[1] = film atoms, out[2] = indenter atoms, out[3] = atom slots (incl. tile padding),
 * out[4] = cells, out[5] = kmax, out[6] = kcmax, out[7] = largest Cr-Cr list length seen at
 * the last rebuild, out[8] = largest Cr-C. */
int md_get_info(md_t *h, int64_t *out9);

/* The last error message of the handle (never NULL; "" when none).  h may be NULL, then
 * the message of the last failed md_init on this thread is returned. */
const char *md_last_error(const md_t *h);

/* Release all device and host memory of the handle (NULL is ignored). */
void md_free(md_t *h);

/* ABI version of this header (incremented on incompatible change). */
int md_version(void);

/* ------------------------------------------------------------ allocation-free evaluation
 *
 * The paper has no counterpart of this call.  It serves callers that must not allocate
 * device memory where they need forces: an engine whose device memory is all held by its
 * own pool allocator, or a per-step loop in which cudaMalloc / cudaFree (which may
 * synchronise the whole device) cannot be afforded.  It evaluates, for one small system
 * and without a handle, the forces and energies that md_init + md_compute_forces give in
 * MD_FP64 mode with params->tabulated = 0: the forms of Eqs. A1-A5 in FP64, summed over
 * all pairs (no cell grid, no Verlet list).
 *
 * Scratch: one static device array inside the library, MD_SMALL_SCRATCH_BYTES long
 * (about 260 KB), holding F'(rho_i), M'(P_i) of every atom and per-block energy sums.  No
 * scratch word has to start at zero: each call writes every word before it reads it.
 * Apart from the set-up below, a call allocates nothing, on the device or on the host,
 * and calls nothing that does (no cudaMalloc / cudaFree, no allocating library routine).
 *
 * Set-up: the first call on a device (the current device at the call) looks up the
 * scratch address (cudaGetSymbolAddress, checked) and loads the three kernels, then
 * caches the address for that device; if the CUDA runtime has not yet been used on that
 * device, this also creates its context.  Make this first call -- n_cr = 0 does only the
 * set-up -- before any stream capture begins.  The cached address belongs to the context
 * the set-up ran in: after cudaDeviceReset on that device (which destroys the context and
 * the array with it) this function must not be called again in the same process.
 *
 * Concurrency: every call on a device uses the same scratch.  Calls whose kernels overlap
 * in time (two streams, or two host threads) race on it and return wrong results; order
 * them on one stream or with events.
 *
 * Arguments.  Arrays marked (dev) are DEVICE pointers owned by the caller, row-major
 * n x 3 doubles in Angstrom; the rest are host pointers.
 *   params            potential; params->tabulated must be 0
 *   n_cr, x_cr (dev)  film atoms, 0 <= n_cr <= MD_SMALL_MAX_ATOMS (0: set-up only)
 *   n_c, x_c (dev)    indenter atoms at their current positions, 0 <= n_c <=
 *                     MD_SMALL_MAX_ATOMS (x_c may be NULL when n_c = 0)
 *   box_lo, box_hi, periodic   3 each; along a periodic axis the length must exceed twice
 *                     the larger cut-off (every pair is taken at its minimum image)
 *   F (dev)           out: force on each film atom (n_cr x 3, eV/A)
 *   energy (dev)      out: 4 doubles, sum_i F(rho_i), sum_{i<j} Phi, sum_i M(P_i),
 *                     sum_{i,c} phi(y_ic) (eV) -- md_energy's embed, pair, mterm, morse
 *   stream            cudaStream_t of the launches (NULL: the legacy default stream)
 *   errbuf, errlen    optional host buffer for the message of a rejected call
 * Returns MD_OK once the kernels are queued (they run asynchronously on stream), else
 * MD_ERR_ARG (a size above the maximum, a bad box or potential: nothing launched) or
 * MD_ERR_CUDA.
 */
#define MD_SMALL_MAX_ATOMS 16384
#define MD_SMALL_SCRATCH_BYTES (8 * (2 * MD_SMALL_MAX_ATOMS + 4 * (MD_SMALL_MAX_ATOMS / 128)))
int md_forces_small(const md_params *params, int32_t n_cr, const double *x_cr, int32_t n_c,
                    const double *x_c, const double box_lo[3], const double box_hi[3],
                    const int32_t periodic[3], double *F, double *energy, void *stream,
                    char *errbuf, size_t errlen);

/* Measurement helper (no counterpart in the paper): the FP64 FMA rate of the current
 * device's CUDA cores, from eight independent FMA chains per thread over 8 CTAs of 256
 * threads per SM, timed with CUDA events; *flops_per_s counts 2 flops per FMA, *ms (may be
 * NULL) is one launch's time.  The FP64 form of the force kernels is bounded by this rate.
 * Allocates and frees its own buffer; synchronises.  Errors: MD_ERR_ARG, MD_ERR_CUDA. */
int md_probe_fp64_fma(double *flops_per_s, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
