/*
 * abfe.h - C ABI of the GB300 alchemical nonbonded engine.
 *
 * The engine evaluates, for many lambda windows ("replicas") of absolute
 * binding free energy (ABFE) legs at once, the alchemical nonbonded forces and
 * energies that dominate the MD sampling of each window, integrates the windows
 * with a BAOAB Langevin step, and emits dU/dlambda and the reduced-potential
 * row u_kn that MBAR consumes.
 *
 * Method (from the paper "Development and large-scale benchmarks of a
 * protein-ligand absolute binding free energy toolkit"):
 *  - Beutler softcore LJ  U = lambda_ij 4 eps_ij (sigma^12/r_eff^12 - sigma^6/r_eff^6),
 *    r_eff^6 = alpha (1 - lambda_ij)^p sigma^6 + r^6, Lorentz-Berthelot mixing,
 *    lambda_ij = min(lambda_i, lambda_j) with environment atoms at 1, applied to
 *    ligand-environment and ligand-ligand pairs (section "Double annihilation
 *    protocol");
 *  - ligand partial charges scaled linearly by lambda_q (same section);
 *  - real-space Ewald (erfc) Coulomb at the PME real-space cutoff (appendix
 *    "Additional methodological details");
 *  - Boresch restraint: distance P1-L1, angles P1-L1-L2 and L1-P1-P2 as
 *    (k/2)(g-g0)^2, dihedrals P2-P1-L1-L2, P1-L1-L2-L3, L1-P1-P2-P3 as
 *    k[1-cos(g-g0)], scaled by lambda_r (section "Restraints");
 *  - u_kn of every frame at all K states for MBAR (section "Simulation protocol").
 *
 * Conventions for every call:
 *  - Units: nm, ps, amu, e, kJ/mol. Boxes are orthorhombic.
 *  - Every call returns an abfe_status; none aborts, traps or exits. After a
 *    failure abfe_last_error() describes it.
 *  - Pointers named h_* are caller-owned HOST memory; inputs are copied before
 *    the call returns, outputs are complete when it returns (the call
 *    synchronises the context's stream). Pointers named d_* are caller-owned
 *    DEVICE memory on the current device; work on them is ordered on the
 *    context's stream.
 *  - The context owns all device memory it allocates (through the allocator
 *    hook if one was installed before abfe_create) and frees it in abfe_destroy.
 *  - Atom indices are per system, 0-based, in the order of the system
 *    description ("original order"). Replica r's atoms occupy rows
 *    [atom_offset(r), atom_offset(r) + n_atoms(r)) of the concatenated
 *    per-atom host arrays, replicas in index order.
 */
#ifndef ABFE_H
#define ABFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct abfe_ctx abfe_ctx;

typedef enum {
    ABFE_OK = 0,
    ABFE_ERR_INVALID_ARG = 1,       /* a NULL pointer, size or value out of range */
    ABFE_ERR_CUTOFF_TOO_LARGE = 2,  /* r_c >= L/2 for some box edge */
    ABFE_ERR_LIST_OVERFLOW = 3,     /* a neighbour-list or cell capacity was exceeded */
    ABFE_ERR_NONFINITE = 4,         /* a non-finite force or energy was produced (reported ahead
                                       of the list overflows it usually causes) */
    ABFE_ERR_CUDA = 5,              /* a CUDA runtime call failed */
    ABFE_ERR_TIMEOUT = 6,           /* a bounded device wait gave up */
    ABFE_ERR_NOT_IMPLEMENTED = 7,
    ABFE_ERR_STATE = 8,             /* call made in the wrong order (e.g. no schedule) */
    ABFE_ERR_OUT_OF_MEMORY = 9
} abfe_status;

/* Energy components written by abfe_compute, per replica (kJ/mol). */
enum {
    ABFE_E_ENV_LJ = 0,     /* environment-environment LJ */
    ABFE_E_ENV_COUL,       /* environment-environment real-space Coulomb */
    ABFE_E_LIGENV_LJ,      /* ligand-environment softcore LJ at lambda_v */
    ABFE_E_LIGLIG_LJ,      /* ligand-ligand LJ (softcore when annihilating) */
    ABFE_E_LIGENV_COUL,    /* ligand-environment Coulomb at lambda_q */
    ABFE_E_LIGLIG_COUL,    /* ligand-ligand Coulomb (x lambda_q^2 when annihilating) */
    ABFE_E_BOND,           /* harmonic bonds (lambda independent) */
    ABFE_E_RESTRAINT,      /* lambda_r * U_Boresch */
    ABFE_E_RECIP,          /* reciprocal + self + excluded-pair Ewald terms at lambda_q (0 without PME) */
    ABFE_E_TORSION,        /* rotatable-bond torsions: lambda_v * U_T (annihilating) or U_T */
    ABFE_E_TOTAL,
    ABFE_N_ENERGY
};

/* dU/dlambda components written per replica (kJ/mol). */
enum { ABFE_DUDL_RESTRAINT = 0, ABFE_DUDL_COUL = 1, ABFE_DUDL_VDW = 2, ABFE_N_DUDL = 3 };

/* One system (one leg's structure). Host memory, copied by abfe_create. */
typedef struct {
    int32_t n_atoms;
    double box[3];                 /* orthorhombic edge lengths, nm */
    const double *pos;             /* [n][3] nm */
    const double *vel;             /* [n][3] nm/ps, or NULL for zero */
    const double *mass;            /* [n] amu (> 0) */
    const double *charge;          /* [n] e */
    const double *sigma;           /* [n] nm (>= 0) */
    const double *epsilon;         /* [n] kJ/mol (>= 0) */
    const uint8_t *is_ligand;      /* [n] 1 = alchemical (ligand) atom */
    int32_t n_excl;
    const int32_t *excl;           /* [n_excl][2] excluded pairs (no nonbonded term) */
    int32_t n_bonds;
    const int32_t *bond_idx;       /* [n_bonds][2] harmonic bonds, may be NULL if 0 */
    const double *bond_r0;         /* [n_bonds] nm */
    const double *bond_k;          /* [n_bonds] kJ/mol/nm^2, U = (k/2)(r-r0)^2 */
    int32_t has_boresch;
    int32_t anchors[6];            /* P1, P2, P3, L1, L2, L3 */
    double b_r0;                   /* nm */
    double b_theta0[2];            /* P1-L1-L2, L1-P1-P2, rad */
    double b_phi0[3];              /* P2-P1-L1-L2, P1-L1-L2-L3, L1-P1-P2-P3, rad */
    double b_kr, b_ktheta, b_kphi; /* kJ/mol/nm^2, kJ/mol/rad^2, kJ/mol */
    /* Periodic torsions of the ligand's rotatable bonds ("Double annihilation
     * protocol": scaled linearly with the alchemical parameter). U = s sum_t
     * k_t [1 + cos(n_t phi_t - phi0_t)], phi_t the dihedral of atoms (a, b, c, d)
     * about b-c (IUPAC sign), s = lambda_v when annihilating (ligand_mode 0) and
     * 1 when decoupling (ligand_mode 1). Arrays may be NULL if n_torsions is 0. */
    int32_t n_torsions;
    const int32_t *torsion_idx;    /* [n_torsions][4] atom indices a, b, c, d (distinct) */
    const double *torsion_k;       /* [n_torsions] kJ/mol */
    const int32_t *torsion_n;      /* [n_torsions] periodicity 1..6 */
    const double *torsion_phi0;    /* [n_torsions] phase, rad */
    /* Alchemical waters ("Double annihilation protocol": the box stays neutral
     * along the path). The oxygen of each carries q + (1 - lambda_q) dq, dq its
     * share of the ligand's net charge (the paper keeps each share within
     * -0.4..0.6 e and their number fixed across windows); forces, energies,
     * dU/dlambda_q and u_kn follow. Arrays may be NULL if n_alch_waters is 0.
     * With pme_order > 0 abfe_create returns ABFE_ERR_NOT_IMPLEMENTED. */
    int32_t n_alch_waters;
    const int32_t *alch_water_idx; /* [n_alch_waters] atom indices: distinct, not ligand atoms */
    const double *alch_water_dq;   /* [n_alch_waters] e */
} abfe_system_desc;

typedef struct {
    double cutoff;        /* r_c, nm: LJ and real-space Coulomb are truncated at r < r_c */
    double ewald_beta;    /* 1/nm; FP32 mode needs ewald_beta * cutoff <= 3.6 */
    double sc_alpha;      /* softcore alpha (paper: 0.5) */
    double sc_p;          /* softcore p (paper: 1) */
    double coulomb_k;     /* kJ mol^-1 nm e^-2 */
    double kT;            /* kJ/mol, for u_kn and the thermostat */
    double skin;          /* nm; list radius r_c + skin, rebuilt when an atom moved > skin/2 */
    int32_t ligand_mode;  /* 0 = annihilate (paper default), 1 = decouple */
    int32_t precision;    /* 0 = FP32 pair arithmetic, 1 = FP64 pair arithmetic */
    /* Reciprocal-space Ewald (smooth PME, Essmann et al. 1995), the rest of the
     * paper's PME electrostatics ("Additional methodological details"):
     * pme_order 0 = real-space Coulomb only; 4, 5 or 6 = B-spline order, with a
     * grid of K = 2^a 3^b 5^c points per box edge, the smallest with
     * L / K <= pme_spacing (nm) and K >= 2 pme_order, K <= 256. Adds the
     * reciprocal energy of the charges at lambda_q, the self energy
     * -k_e beta / sqrt(pi) sum q^2 and the excluded-pair correction
     * -k_e sum q_i q_j erf(beta r)/r to forces, energies (ABFE_E_RECIP), dU/dlambda_q
     * and u_kn. Grid and FFT in FP32, energy sums in FP64, in both precision
     * modes. Needs ligand_mode 0 (ABFE_ERR_NOT_IMPLEMENTED otherwise). */
    double pme_spacing;
    int32_t pme_order;
    int32_t pme_reserved; /* 0 */
} abfe_params;

/* Launch shape of the pair kernels (chosen by abfe_autotune or set by hand). */
typedef struct {
    int32_t group;          /* i-clusters of 8 atoms per outer-list group (one candidate search
                               and one prune work item): 1, 2 or 4 */
    int32_t max_entries;    /* j-clusters per outer work item before a list is split: 16..512 */
    int32_t block_threads;  /* threads per block of the environment pair kernel: 64..256,
                               multiple of 32 */
    int32_t graph_steps;    /* steps per captured CUDA graph (0 = launch kernels directly) */
    double skin;            /* nm: outer list radius r_c + skin, rebuilt when an atom may have
                               moved > skin/2 since the build (0 <= skin <= max(params.skin,
                               0.3)) */
    double prune_skin;      /* nm: inner (pruned) list radius r_c + prune_skin, re-pruned from
                               the outer list when an atom moved > prune_skin/2 since the
                               last prune (0 <= prune_skin <= min(skin, 0.15)) */
    int32_t reserved0;      /* 0 */
    int32_t reserved1;      /* 0 */
} abfe_tuning;

/* Device time of the pair kernels, from CUDA events recorded on the context's
 * stream around each launch while profiling is on. A launch inside a CUDA
 * graph keeps the duration of its most recent replay. */
typedef struct {
    double env_ms;            /* summed duration of environment pair-kernel launches */
    int64_t env_launches;
    double lig_ms;            /* summed duration of ligand pair-kernel launches */
    int64_t lig_launches;
    double integrate_ms;      /* summed duration of integrator launches */
    int64_t integrate_launches;
    double build_ms;          /* outer list builds that the host forces (abfe_build_neighbor_list,
                                 a tuning change): cell list, sort and cluster-pair list */
    int64_t build_launches;
    double prune_ms;          /* prunes of the inner list that the host forces (with every forced
                                 build) */
    int64_t prune_launches;
} abfe_profile;

typedef struct {
    int64_t n_items_env, n_items_lig;     /* work items of the last list build */
    int64_t n_entries, n_xentries;        /* cluster-pair entries (plain, with exclusion masks) */
    int64_t n_rebuilds;                   /* outer-list build events (any window) since create */
    int64_t steps_done;
    int64_t slots, clusters;              /* padded atom slots and clusters (all replicas) */
    int64_t device_bytes;                 /* device memory held by the context */
    int64_t env_lane_groups;              /* pair lanes the environment kernel computes over
                                             the inner list, divided by 32 (a warp round of
                                             32 rows counts 4 for each half block of i atoms
                                             it evaluates), from the last abfe_count_pairs */
    int64_t n_prunes;                     /* inner-list prune events (any window) since create */
    int64_t n_rows, n_xrows;              /* inner-list rows (plain, with excluded pairs) */
    int64_t n_exchange_attempts;          /* abfe_replica_exchange calls since create (or as
                                             restored by a checkpoint) */
    int64_t n_exchange_accepted;          /* accepted state swaps since create */
    int64_t n_window_rebuilds;            /* windows rebuilt, summed over the build events */
    int64_t n_window_prunes;              /* windows pruned, summed over the prune events */
} abfe_stats;

/* Optional device allocator (e.g. PyTorch's caching allocator). Install before
 * abfe_create; the hook is global to the library. alloc returns NULL on
 * failure; stream is the context's cudaStream_t. */
typedef void *(*abfe_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*abfe_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
void abfe_set_allocator(abfe_alloc_fn alloc_fn, abfe_free_fn free_fn, void *user);

/* Create a context for n_replicas windows. systems[0..n_systems) are the
 * distinct structures; replica r simulates systems[system_of_replica[r]]
 * (replicas of one system start from identical coordinates). cuda_stream is a
 * cudaStream_t (NULL = legacy default stream). Fails with
 * ABFE_ERR_CUTOFF_TOO_LARGE if r_c >= L/2, ABFE_ERR_INVALID_ARG for bad
 * indices, parameters or sizes. */
abfe_status abfe_create(const abfe_system_desc *systems, int32_t n_systems,
                        const int32_t *system_of_replica, int32_t n_replicas,
                        const abfe_params *params, void *cuda_stream, abfe_ctx **out);

/* Register lambda schedule `schedule_id` (0..15) with K states (1..256):
 * lam_r[k] (restraint, 0 = off), lam_q[k] (ligand charge scale), lam_v[k]
 * (softcore coupling), each in [0, 1]. Host arrays, copied. */
abfe_status abfe_set_lambda_schedule(abfe_ctx *ctx, int32_t schedule_id, int32_t K,
                                     const double *lam_r, const double *lam_q,
                                     const double *lam_v);

/* Assign each replica a schedule and a state index in it (host arrays of
 * length n_replicas). Must be called before compute/step/eval. */
abfe_status abfe_set_replica_states(abfe_ctx *ctx, const int32_t *schedule_of_replica,
                                    const int32_t *state_of_replica);

/* Rebuild the cell list and cluster-pair list from the current positions. */
abfe_status abfe_build_neighbor_list(abfe_ctx *ctx);

/* Forces and energies of every replica at its own state and current
 * positions. h_forces: [total_atoms][3] kJ/mol/nm in original order or NULL;
 * h_energy: [R][ABFE_N_ENERGY] or NULL; h_dudl: [R][ABFE_N_DUDL] or NULL. */
abfe_status abfe_compute(abfe_ctx *ctx, double *h_forces, double *h_energy, double *h_dudl);

/* Same evaluation with device outputs: d_forces [total_atoms][3] float
 * (original order) or NULL, d_energy [R][ABFE_N_ENERGY] double or NULL,
 * d_dudl [R][ABFE_N_DUDL] double or NULL. Stream-ordered, no host sync. */
abfe_status abfe_compute_device(abfe_ctx *ctx, float *d_forces, double *d_energy, double *d_dudl);

/* Advance every replica by n_steps BAOAB Langevin steps (B A O A, forces, B)
 * of length dt (ps) with friction gamma (1/ps) at kT. Random normals come from
 * Philox4x32-10 with counter (atom index, step low, step high, replica) and key
 * (seed low, seed high), converted by Box-Muller. The list is rebuilt inside
 * the step whenever an atom moved more than skin/2 since the last build. */
abfe_status abfe_step(abfe_ctx *ctx, int32_t n_steps, double dt, double gamma, uint64_t seed);

/* Reduced potentials of the current frame: h_ukn[r][k] = U_k(x_r)/kT for every
 * state k of replica r's schedule (row stride ld >= max K; unused entries 0).
 * h_du (optional, same shape, kJ/mol) gets the lambda-dependent part
 * U_k - U_indep, where U_indep (the environment pairs, bonds and, when
 * decoupling, the ligand's own pairs) is the same at every state. h_dudl
 * (optional, [R][3]) gets dU/dlambda at each replica's own state. */
abfe_status abfe_eval_ukn(abfe_ctx *ctx, double *h_ukn, double *h_du, int32_t ld,
                          double *h_dudl);

/* Positions / velocities of all replicas, original order, [total_atoms][3]. */
abfe_status abfe_get_positions(abfe_ctx *ctx, double *h_pos);
abfe_status abfe_set_positions(abfe_ctx *ctx, const double *h_pos);
abfe_status abfe_get_velocities(abfe_ctx *ctx, double *h_vel);
abfe_status abfe_set_velocities(abfe_ctx *ctx, const double *h_vel);

/* Number of in-cutoff non-excluded pairs found through the cluster list:
 * h_counts[r][0] environment-environment, h_counts[r][1] ligand-involved, and
 * (optional) h_atom_counts[total_atoms]: partners of each atom. */
abfe_status abfe_count_pairs(abfe_ctx *ctx, int64_t *h_counts, int32_t *h_atom_counts);

abfe_status abfe_set_tuning(abfe_ctx *ctx, const abfe_tuning *t);
abfe_status abfe_get_tuning(abfe_ctx *ctx, abfe_tuning *t);
/* Time candidate tunings on the context's own replicas and keep the fastest.
 * cache_path (may be NULL) is a JSON file of earlier results keyed by the
 * workload's shape; a hit skips the search. */
abfe_status abfe_autotune(abfe_ctx *ctx, const char *cache_path, int32_t reps);
/* Pick the outer skin (rebuild cadence) and the prune skin (prune cadence)
 * that minimise the modelled time per MD step. It measures D(n), the largest
 * displacement of any atom n steps after an outer build, over up to n_steps
 * (default 48 when n_steps < 8) steps of (dt, gamma, seed); then for every
 * candidate pair, skin in {0.1, 0.15, 0.2, 0.25, 0.3} nm (up to the cap) and
 * prune_skin in {0.02, 0.04, 0.06, 0.1, 0.15} nm (<= skin), it times one forced
 * build B(skin), one forced prune P(skin, prune_skin) and one pair pass
 * E(prune_skin). A rebuild comes every n_b steps, the first n with
 * D(n) > skin/2, and a prune every n_p steps, D(n) > prune_skin/2, plus one
 * with each rebuild. The cost per step is
 * E + (B + ceil(n_b / n_p) P) / n_b. The measurement runs from a saved state
 * that is restored afterwards, so the trajectory is the one without the tuner. */
abfe_status abfe_autotune_cadence(abfe_ctx *ctx, double dt, double gamma, uint64_t seed,
                                  int32_t n_steps);
abfe_status abfe_get_stats(abfe_ctx *ctx, abfe_stats *s);

/* Replica exchange within each segment (the paper confines exchange to the
 * windows that one GPU hosts, "Simulation protocol"). An exchange group is the
 * set of replicas that share a system and a schedule; its states must be
 * distinct. Attempt t (the t-th attempt since create, counting abfe_step's
 * in-loop attempts) pairs the replicas holding
 * neighbouring states of the group - positions (m, m+1) of its states in
 * ascending order, m = t mod 2, t mod 2 + 2, ... - and swaps their states with
 * probability min(1, exp(-D)), D = u_b(x_ra) + u_a(x_rb) - u_a(x_ra) - u_b(x_rb)
 * (reduced potentials; ra held state a, rb held b), decided in FP64 on the
 * device. The uniform is Philox4x32-10 at counter (t & 0xffffffff, t >> 32,
 * group, m) with key (seed & 0xffffffff, seed >> 32): with words x0, x1,
 * U = ((x0 >> 5) * 2^26 + (x1 >> 6) + 0.5) * 2^-53, accept iff D <= 0 or
 * ln U < -D. Coordinates and velocities stay with their replica; forces are
 * recomputed at the next step.
 *  - h_ukn: NULL to evaluate the u_kn rows on the device at the current
 *    coordinates (as abfe_eval_ukn), else host [R][ld] reduced potentials to
 *    decide with (entries k >= K of a replica's schedule are ignored).
 *  - h_ukn_out: host [R][ld] or NULL: the rows used (when evaluated here).
 *  - h_state: host [R] or NULL: every replica's state after the attempt.
 *  - h_n_accepted: host or NULL: swaps accepted in this attempt.
 * Errors: ABFE_ERR_STATE (states not set, or a group holds a state twice),
 * ABFE_ERR_INVALID_ARG (ld < K), ABFE_ERR_NONFINITE (non-finite h_ukn entry). */
abfe_status abfe_replica_exchange(abfe_ctx *ctx, uint64_t seed, const double *h_ukn, int32_t ld,
                                  double *h_ukn_out, int32_t *h_state, int32_t *h_n_accepted);
/* Current state index of every replica (after device-side exchanges), host [R]. */
abfe_status abfe_get_replica_states(abfe_ctx *ctx, int32_t *h_state);
/* Replica exchange inside the step loop ("Simulation protocol": exchanges among
 * one GPU's windows every 5 ps). With every_steps > 0, abfe_step attempts one
 * exchange (the rule of abfe_replica_exchange, attempt numbers continuing
 * theirs, key `seed`) at the end of every step whose device step count is a
 * multiple of every_steps, entirely on the device: the step's closing half
 * kick, the u_kn rows of all replicas at the current coordinates, the
 * exchange, forces for the new states and the half kick that opens the next
 * step. In a captured step graph this is a conditional node (no host round
 * trip); direct launches give the same trajectory bit for bit. 0 switches it
 * off. Errors: ABFE_ERR_INVALID_ARG (every_steps < 0), ABFE_ERR_STATE (states
 * not set, or a group holds a state twice). */
abfe_status abfe_set_exchange(abfe_ctx *ctx, int32_t every_steps, uint64_t seed);
/* Profiling: max_launches > 0 allocates that many event pairs per kernel kind
 * and starts recording (counts reset); 0 stops. abfe_get_profile synchronises
 * and sums the recorded durations. */
abfe_status abfe_set_profiling(abfe_ctx *ctx, int32_t max_launches);
abfe_status abfe_get_profile(abfe_ctx *ctx, abfe_profile *p);

/* Checkpoint: positions, velocities, step counter, seed and replica states
 * (binary file). Resuming continues the same trajectory bit for bit. */
abfe_status abfe_save_checkpoint(abfe_ctx *ctx, const char *path);
abfe_status abfe_load_checkpoint(abfe_ctx *ctx, const char *path);

/* ---------------------------------------------------------------------------
 * Entry point that allocates nothing. The paper has no counterpart: it exists
 * for callers that cannot allocate device memory themselves, for example a
 * plugin running inside a host MD engine or application whose device memory is
 * owned by the host's own allocator or fixed budget. It needs no context.
 *
 * abfe_ukn_frame_noalloc writes, for one frame of one window, the
 * lambda-dependent part of the reduced-potential row in kJ/mol: for every
 * state k, the ligand pairs inside the cutoff at (lambda_q,k, lambda_v,k)
 * (Beutler LJ and real-space Ewald Coulomb) plus lambda_r,k times the Boresch
 * energy, in FP64 arithmetic. It covers real-space Coulomb only and has no
 * torsion or alchemical-water input: it equals what abfe_eval_ukn returns in
 * h_du for a context created with pme_order = 0 whose systems have neither
 * rotatable-bond torsions nor alchemical waters (not the reciprocal, self and
 * excluded-pair terms that pme_order > 0 adds, nor the lambda_v,k U_T torsion
 * term or the alchemical waters' charge terms, which the caller adds if it has
 * them).
 *  - Inputs are device arrays on the current device (FP32 coordinates and
 *    parameters, original atom order); schedule, box, restraint and parameters
 *    are host values inside the struct. The caller owns inputs and output.
 *  - d_du: device array of K doubles, written in stream order on cuda_stream.
 *  - Scratch is a file-scope __device__ array of ABFE_NOALLOC_MAX_BLOCKS x
 *    (ABFE_NOALLOC_MAX_K + 2) doubles (about 1 MB) that every GPU loading the
 *    library holds until the process exits. Every call shares it and it keeps
 *    the last call's contents (each call overwrites what it reads): calls that
 *    overlap on the GPU race with each other and must be ordered by the caller.
 *  - The first call on a device looks up the scratch array's device address
 *    with cudaGetSymbolAddress (that device current); make that first call
 *    before any stream capture. No call allocates or frees device memory.
 *  - Sizes beyond the maxima below return ABFE_ERR_INVALID_ARG before any
 *    launch. lig_excl holds at most ABFE_NOALLOC_MAX_EXCL partners per ligand
 *    atom; the call sees only those, so a system with a ligand atom that has
 *    more excluded partners must be rejected by the caller (the pairs left out
 *    of lig_excl would be counted as ordinary pairs).
 *  - Device data are not validated on the host: a lig_idx entry outside
 *    [0, n_atoms) is never dereferenced; it turns every du[k] of that call
 *    into NaN. Anchor indices (host values) are checked.
 *  - Cost: every ligand atom scans all n_atoms atoms once per 16 states
 *    (ceil(K / 16) passes); one call is n_lig x ceil(K / 16) x n_atoms pair
 *    tests in FP64.
 */
#define ABFE_NOALLOC_MAX_ATOMS (1 << 22)
#define ABFE_NOALLOC_MAX_LIG 1024
#define ABFE_NOALLOC_MAX_K 128
#define ABFE_NOALLOC_MAX_EXCL 16
#define ABFE_NOALLOC_MAX_BLOCKS 1024

typedef struct {
    int32_t n_atoms;                 /* <= ABFE_NOALLOC_MAX_ATOMS */
    double box[3];                   /* nm */
    const float *pos;                /* device [n][3] nm */
    const float *charge;             /* device [n] e */
    const float *sigma;              /* device [n] nm */
    const float *epsilon;            /* device [n] kJ/mol */
    const uint8_t *is_ligand;        /* device [n] */
    int32_t n_lig;                   /* <= ABFE_NOALLOC_MAX_LIG */
    const int32_t *lig_idx;          /* device [n_lig] atom index of each ligand atom */
    const int32_t *lig_excl;         /* device [n_lig][ABFE_NOALLOC_MAX_EXCL] excluded partners, -1 padded */
    int32_t K;                       /* states, <= ABFE_NOALLOC_MAX_K */
    double lam_r[ABFE_NOALLOC_MAX_K], lam_q[ABFE_NOALLOC_MAX_K], lam_v[ABFE_NOALLOC_MAX_K];
    double cutoff, ewald_beta, sc_alpha, sc_p, coulomb_k;
    int32_t ligand_mode;             /* 0 annihilate, 1 decouple */
    int32_t has_boresch;
    int32_t anchors[6];
    double b_r0, b_theta0[2], b_phi0[3], b_kr, b_ktheta, b_kphi;
} abfe_noalloc_frame;

abfe_status abfe_ukn_frame_noalloc(const abfe_noalloc_frame *frame, double *d_du, void *cuda_stream);

/* ---------------------------------------------------------------------------
 * MBAR free energies of the states of one window segment (Shirts & Chodera
 * 2008). The paper estimates the free-energy difference between the terminal
 * states of each GPU segment with MBAR and sums the segments ("Simulation
 * protocol"); this is that estimator. No context is needed.
 *
 * Solves f_i = -ln sum_n exp(-u_in) / sum_k N_k exp(f_k - u_kn), f_0 = 0, by
 * self-consistent iteration in FP64 until max_k |f_k(t+1) - f_k(t)| < tol, or
 * max_iter iterations. Every iteration runs on the device; the loop is one
 * CUDA graph with a conditional while node (a host loop where the driver lacks
 * conditional nodes). Results are deterministic.
 *  - u_kn: [K][N] row major, u_kn[k * N + n] = reduced potential (energy / kT)
 *    of sample n at state k. Samples are ordered by the state that drew them:
 *    the first N_0 from state 0, the next N_1 from state 1, ... abfe_mbar reads
 *    host memory; abfe_mbar_device reads device memory, ordered after the work
 *    already queued on `stream` (NULL: the legacy default stream).
 *  - N_k: [K] host, N_k >= 0, sum N_k = N. States with N_k = 0 receive their
 *    free energy without contributing samples.
 *  - f_k: [K] host output, dimensionless (kT units), f_0 = 0.
 *  - n_iter: host output (may be NULL), iterations done; == max_iter means the
 *    tolerance was not reached (status is still ABFE_OK).
 *  - Errors: ABFE_ERR_INVALID_ARG (NULL pointers, K < 1 or K > ABFE_MBAR_MAX_K,
 *    N < 1, a negative N_k or sum N_k != N, tol <= 0, max_iter < 1);
 *    ABFE_ERR_NONFINITE (a non-finite u_kn or free energy); ABFE_ERR_OUT_OF_MEMORY;
 *    ABFE_ERR_CUDA. The message is abfe_last_error(NULL).
 *  - Device scratch of about 8 (K N + N + 2 K N / 16384 + 4 K) bytes, plus
 *    8 K N bytes for the copy of u_kn in abfe_mbar, comes from the allocator
 *    installed by abfe_set_allocator (else cudaMalloc) and is freed on return.
 */
#define ABFE_MBAR_MAX_K 1024
abfe_status abfe_mbar(const double *h_u_kn, const int32_t *h_N_k, int32_t K, int64_t N,
                      double tol, int32_t max_iter, double *h_f_k, int32_t *h_n_iter);
abfe_status abfe_mbar_device(const double *d_u_kn, const int32_t *h_N_k, int32_t K, int64_t N,
                             double tol, int32_t max_iter, double *h_f_k, int32_t *h_n_iter,
                             void *stream);

/* ---------------------------------------------------------------------------
 * Standard-state correction of the Boresch restraint ("Restraints": the free
 * energy of the restraints in the decoupled state, added analytically to the
 * simulated legs; the paper cites the expression without printing it). Returns
 * in *dG (kJ/mol) the free energy of imposing the distance, two angle and
 * three dihedral terms (k_r/2 (r-r0)^2, k_theta/2 (theta-theta0)^2,
 * k_phi [1 - cos(phi-phi0)]) on the decoupled ligand at 1 mol/L:
 *     dG = -kT ln( Z_r Z_thetaA Z_thetaB Z_phi^3 / (8 pi^2 V0) ),
 * V0 = 1.66054 nm^3, from the exact one-dimensional integrals of the
 * factorised restraint partition function (Jacobian r^2 sin(thetaA)
 * sin(thetaB)); the dihedral references drop out. Host computation, no
 * context or device needed. Errors: ABFE_ERR_INVALID_ARG (NULL pointers,
 * kT, r0 or a force constant <= 0, theta0 outside (0, pi)); message in
 * abfe_last_error(NULL). theta0: host [2] (L1 angle P1-L1-L2, P1 angle L1-P1-P2). */
abfe_status abfe_boresch_correction(double kT, double r0, const double *theta0, double k_r,
                                    double k_theta, double k_phi, double *dG);

int32_t abfe_num_replicas(const abfe_ctx *ctx);
int64_t abfe_total_atoms(const abfe_ctx *ctx);
int64_t abfe_atom_offset(const abfe_ctx *ctx, int32_t replica);
const char *abfe_last_error(const abfe_ctx *ctx);
const char *abfe_status_string(abfe_status s);
void abfe_destroy(abfe_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ABFE_H */
