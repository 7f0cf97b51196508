// Internal data layout of the GB300 alchemical nonbonded engine.
//
// All replicas (lambda windows) live in one set of device arrays:
//  * "slots": per-atom arrays in spatially sorted order, grouped in clusters of
//    8 consecutive slots. Replica r owns the fixed cluster range
//    [cl_off, cl_off + n_cl_cap); padding slots are dummies (orig = -1).
//  * Columns: each replica's box is cut into ncx x ncy columns along z plus one
//    ligand column. At every list build the atoms are binned into columns,
//    sorted by z inside each column and cut into clusters of 8; the ligand's
//    atoms get their own clusters, so every cluster pair is either
//    environment-environment (lambda independent, plain LJ + erfc) or
//    ligand-involved (softcore, charge scaling, dU/dlambda, u_kn).
//  * Outer cluster-pair list (radius r_c + skin, rebuilt when an atom may have
//    moved more than skin/2 since the build): a work item is a group of up to 4
//    consecutive i-clusters of one column and a range of j-cluster entries
//    (int2: j cluster, packed half-tile mask | shift | flags). Entries that
//    contain excluded pairs or the cluster's own triangle carry 64-bit masks per
//    i-cluster.
//  * Inner list of j rows (radius r_c + prune_skin, one region per replica,
//    re-pruned from the outer list for each replica one of whose atoms moved
//    more than prune_skin/2 since its last prune): per
//    i-cluster, the j atoms with at least one of the cluster's 8 atoms inside
//    the inner radius, as 32-bit words (j slot | periodic image code), full
//    rows first, then rows with only the cluster's lower or only its upper
//    four atoms in range; rows that contain excluded pairs carry an 8-bit mask
//    of the excluded i atoms. The environment pair kernel walks these rows.
//  * Forces are 64-bit fixed point (2^32 units per kJ/mol/nm) accumulated
//    with integer atomics, so results do not depend on the order of work;
//    energies use the same fixed point per replica.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "abfe.h"
#include "erfc_coeffs.h"

namespace abfe {

constexpr int CL = 8;       // atoms per cluster
constexpr int GMAX = 4;     // i-clusters per work item (max)
constexpr int KV_MAX = 64;  // distinct lambda_v values per replica for u_kn
constexpr int MAX_SCHED = 16;
constexpr int K_MAX = 256;
// Real-space Ewald force table: G(r) = erfc(beta r) + (2 beta / sqrt pi) r
// exp(-beta^2 r^2), so that the Coulomb force on a pair is qq G(r) / r^3 times
// the separation vector. EW_NT points on r in [0, r_c]; point j holds
// (G, G' h, G'' h^2 / 2) at r_j = j h for a centred quadratic in the offset.
constexpr int EW_NT = 1024;
constexpr int COL_MAX = 1024;       // atoms per column (per-column sort capacity)
constexpr double FSCALE = 4294967296.0;
constexpr float FSCALEF = 4294967296.0f;
constexpr double INV_FSCALE = 1.0 / 4294967296.0;
constexpr float DUMMY_FAR = 1.0e4f;

// error bits (Counters::err)
enum : int {
    ERRB_LIST = 1,        // entry / item capacity exceeded
    ERRB_NONFINITE = 2,   // NaN / inf force or energy
    ERRB_COLUMN = 4,      // a column exceeded COL_MAX atoms
    ERRB_CLUSTERS = 8,    // a replica exceeded its cluster capacity
    ERRB_GROUP = 16,      // an i-group exceeded its per-warp entry or mask capacity
    ERRB_INDEX = 32,      // inconsistent index (defensive check)
};

// which capacity an ERRB_LIST overflow hit: err_info[1] = (replica << 4) | kind,
// err_info[2] = the count the region needed (err_info[0] = the i cluster)
enum : int {
    OVF_ENTRIES = 1,      // outer-list entries of the replica's region
    OVF_XENTRIES = 2,     // masked outer-list entries
    OVF_ITEMS_ENV = 3,    // environment work items
    OVF_ITEMS_LIG = 4,    // ligand work items
    OVF_PRUNE_ITEM = 5,   // one outer item above the prune's shared-memory capacity
    OVF_ROWS = 6,         // inner-list rows
    OVF_XROWS = 7,        // masked inner-list rows
    OVF_RITEMS = 8,       // inner-list row items
};

// fixed-point energy accumulator slots per replica
enum : int {
    EA_ENV_LJ = 0, EA_ENV_C, EA_LIGENV_LJ, EA_LIGLIG_LJ, EA_LIGENV_C, EA_LIGLIG_C,
    EA_BOND, EA_DUDLV, EA_DUDLQ,
    // reciprocal space (PME): own-state reciprocal and excluded-pair energies; the
    // lambda_q decomposition A + lambda B + lambda^2 C of the reciprocal energy
    // (A environment, B cross, C ligand) and the excluded pairs by kind
    EA_REC, EA_EXCL, EA_REC_ENV, EA_REC_LIG, EA_REC_MIX, EA_EXCL_ENV, EA_EXCL_MIX, EA_EXCL_LIG,
    EA_TORS,   // unscaled rotatable-bond torsion energy U_T
    // alchemical waters (charge q0 + (1 - lambda_q) dq on their oxygens): with
    // f = k_e erfc(beta r) / r over the oxygens a, A2 = sum dq_a q_j f (j not
    // ligand, not an alchemical oxygen), B2 = sum dq_a q_j f (j ligand, base
    // charge), C01 = sum_{a<b} (q0_a dq_b + dq_a q0_b) f, C11 = sum_{a<b} dq_a dq_b f
    EA_AW_A2, EA_AW_B2, EA_AW_C01, EA_AW_C11,
    EA_N
};

// entry packing: y = half-tile mask (bits 0-7: bit 2g+h = rows 4h..4h+3 of
// i-cluster g against the whole j cluster) | sx+1 (bits 8-9) | sy+1 (bits 10-11)
// | sz+1 (bits 12-13) | j-is-ligand (bit 14); the j cluster is shifted by
// (sx Lx, sy Ly, sz Lz). Rows 0-3 and 4-7 of a cluster are its lower and upper
// z halves, so most cluster pairs have one live half only.
__host__ __device__ __forceinline__ int pack_entry_y(int imask, int sx, int sy, int sz, int jlig) {
    int h = 0;
    for (int g = 0; g < 4; ++g)
        if ((imask >> g) & 1) h |= 3 << (2 * g);
    return h | ((sx + 1) << 8) | ((sy + 1) << 10) | ((sz + 1) << 12) | (jlig << 14);
}
constexpr int ENTRY_SHIFT_BITS = 0x3F00;
constexpr int ENTRY_NOSHIFT = (1 << 8) | (1 << 10) | (1 << 12);
__host__ __device__ __forceinline__ bool entry_half(int y, int g, int h) {
    return (y >> (2 * g + h)) & 1;
}
__host__ __device__ __forceinline__ bool entry_g(int y, int g) { return (y >> (2 * g)) & 3; }
__host__ __device__ __forceinline__ int entry_jlig(int y) { return (y >> 14) & 1; }

struct alignas(16) dbl4 {
    double x, y, z, w;
};

struct RepDev {
    int cl_off, n_cl_cap;          // first cluster, cluster capacity
    int atom_off;                  // offset in the replica-concatenated original-order arrays
    int n_atoms, n_lig;
    int sys;                       // system index
    int sys_atom_off;              // offset in per-system atom arrays
    int sys_ex_off;                // offset of this system's CSR row pointers
    int col_off, ncx, ncy;         // ncx*ncy environment columns + 1 ligand column
    float box[3];
    float colw_inv[2];             // ncx / Lx, ncy / Ly
    int sched, state;
    float lam_q, lam_v, lam_r;
    float sc_A, sc_dA;             // alpha (1-lam_v)^p and d/dlam_v of it
    double dlam_q, dlam_v, dlam_r;
    double dsc_A, dsc_dA;
    int bond_off, n_bonds;         // this system's bonds
    int boresch;                   // index into the Boresch table or -1
    int kv;                        // number of distinct lambda_v in the schedule
    int tors_off, n_tors;          // this system's rotatable-bond torsions
    int aw_off, n_aw;              // this system's alchemical waters
    int n_bond_tri;                // bonded triangles at the head of its bonds
};

struct BoreschDev {
    int anc[6];
    double r0, th0[2], ph0[3], kr, kth, kph;
};

struct Item {
    int c0, ng, rep, e_begin, e_cnt, x_begin, x_cnt, flags;
};

// Inner-list work item: the j rows of one i-cluster from one outer work item
// (the replica is rep_of_cl[c]). Its plain rows start at r_begin in three
// runs: cnt & 0xFFFF full rows (both halves of the i-cluster in range), then
// n_lo rows with only atoms 0-3 in range, then n_hi rows with only atoms 4-7.
// Its masked rows (cnt >> 16 of them) start at x_begin.
struct alignas(16) RowItem {
    int c;
    unsigned int r_begin;
    int x_begin, cnt;
    int n_lo, n_hi, pad0, pad1;
};
// row word: j slot (bits 0-26) | image code (bits 27-31), code = (sx+1) + 3 (sy+1)
// + 9 (sz+1) for the j atom shifted by (sx Lx, sy Ly, sz Lz); 13 = no shift
constexpr int ROW_SLOT_BITS = 27;
constexpr unsigned int ROW_SLOT_MASK = (1u << ROW_SLOT_BITS) - 1u;
constexpr int ROW_NOSHIFT = 13;

struct Counters {
    int env_next, lig_next;        // work-stealing counters of the persistent kernels
    int n_items_env, n_items_lig;
    int n_entries, n_xentries;
    int rebuild;                   // 1 = rebuild the list in this step
    unsigned int maxdisp2;         // float bits of this step's largest squared displacement
                                   // of any atom from its replica's prune positions
    unsigned long long step;       // Langevin step counter (RNG counter)
    int err;
    int err_info[3];
    int n_rebuilds;
    int build_next;                // work counter of the list builder (cluster chunks)
    int prune;                     // 1 = re-prune the inner list in this step
    unsigned int dispb2;           // float bits: max squared displacement of this step's
                                   // positions from the outer build's positions
    unsigned int last_dispb2;      // dispb2 of the last finished step (read by the
                                   // cadence tuner)
    unsigned int n_rows;           // inner list sizes
    int n_xrows, n_ritems;
    int prune_next;                // work counter of the prune kernel (outer items)
    int n_prunes;
    unsigned long long n_win_rebuilds, n_win_prunes;   // windows rebuilt / pruned, summed
    unsigned long long ex_attempt; // replica-exchange attempts so far (the RNG counter)
    long long ex_accepted;         // accepted swaps so far
};

struct StepParams {
    float kick;          // velocity kick factor (ps) applied with F/m
    float half_dt;       // dt/2 (ps) for the two A half-drifts
    float c1;            // exp(-gamma dt)
    float c2;            // sqrt((1 - c1^2) kT)
    unsigned long long seed;
    int drift;           // 1 = A O A after the kick
    int zero_force;      // 1 = clear the force accumulators after reading them
};

struct DevPtrs {
    // replicas
    const RepDev* reps;
    int R;
    const int* rep_of_cl;          // [C] replica of each cluster
    int S, C, NCOL;
    // slot arrays
    float4* xq;                    // x, y, z, q*sqrt(k_e)
    float4* v;                     // vx, vy, vz, 1/m
    float2* se;                    // sigma/2, 2 sqrt(eps)
    int* orig;                     // original atom index in its replica, -1 = dummy
    float4* xref;                  // positions at the last prune (displacement reference)
    float4* xbuild;                // positions at the last outer list build
    long long* fx; long long* fy; long long* fz;
    int* slot_of;                  // [total atoms] slot of each original atom
    // rebuild scratch
    float4* xq_old; float4* v_old; int* orig_old;
    int* slot_col;                 // [S] column of each old slot
    int* perm;                     // [S] new slot -> old slot (-1 dummy)
    int* col_atoms;                // [S] old slots grouped by column
    // columns
    const int* col_rep;            // [NCOL] replica of each column
    int* col_cnt; int* col_fill; int* col_start; int* col_cl_start; int* col_ncl;
    int* cl_col;                   // [C] column of each cluster (-1 unused)
    float4* bbc; float4* bbh;      // cluster bounding box centre / half extent (.w<0: empty)
    float2* clz;                   // cluster z bounds (min, max) of the last build
    // per-system data
    const float4* sys_prm;         // q sqrt(ke), sigma/2, 2 sqrt(eps), 1/m
    const dbl4* sys_prmd;         // q, sigma, eps, 1/m  (FP64 path)
    const unsigned char* sys_lig;
    const int* sys_ex_off;
    const int* sys_ex_idx;
    const int2* sys_bond;
    const float2* sys_bond_p;      // r0, k
    const int* bond_pref;          // bonds of replicas before r (R + 1 entries)
    const int* bond_blk_rep;       // replica of the first bond of each 256-bond block
    int n_bond_total;              // bonds of all replicas
    const BoreschDev* bor;
    const int4* sys_tors;          // torsion atoms a, b, c, d (original indices)
    const dbl4* sys_torsp;         // k, n, phi0, -
    const int* sys_aw;             // alchemical oxygens (original indices), per system
    const float* sys_dq;           // per system atom: dq sqrt(k_e) (0 unless an alchemical oxygen)
    const double* sys_dqd;         // the same in e, FP64
    int has_aw;                    // 1 = some system has alchemical waters
    // lists
    Item* items_env; Item* items_lig;
    int cap_items_env, cap_items_lig;
    int2* entries; int cap_entries;
    int2* xentries; unsigned long long* xmasks; int cap_xentries;
    unsigned int* rows; unsigned int cap_rows;   // inner list: plain j rows
    int2* xrows; int cap_xrows;         // inner list: (row word, excluded i atoms) rows
    RowItem* ritems; int cap_ritems;
    // the inner list in one region per replica (pruned per replica): region
    // bases and capacities, fill counts, and the prefix of the replicas' item
    // counts over which the pair kernels iterate
    const unsigned int* row_base; const unsigned int* row_cap;
    const int* xrow_base; const int* xrow_cap;
    const int* ritem_base; const int* ritem_cap;
    unsigned int* n_rows_r; int* n_xrows_r; int* n_ritems_r;
    int* ritem_pref;               // [R + 1]
    int* ritem_blk;                // replica of item 256 b, for every block b of items
    unsigned int* disp_r;          // float bits: this step's largest squared displacement
                                   // from the replica's prune positions
    int* pflag;                    // 1: the replica is pruned in this step
    // the outer list in one region per replica (rebuilt per replica): entries,
    // masked entries (and their masks), environment and ligand work items
    const int* ent_base; const int* ent_cap; const int* xent_base; const int* xent_cap;
    const int* ienv_base; const int* ienv_cap; const int* ilig_base; const int* ilig_cap;
    int* n_entries_r; int* n_xentries_r; int* n_items_env_r; int* n_items_lig_r;
    int* ienv_pref; int* ilig_pref;  // [R + 1] prefixes of the item counts
    unsigned int* dispb_r;         // float bits: this step's largest squared displacement
                                   // from the replica's outer-build positions
    int* bflag;                    // 1: the replica's outer list is rebuilt in this step
    // outputs
    long long* eacc;               // [R][EA_N]
    double* eb;                    // [R] unscaled Boresch energy
    long long* ukn_lj;             // [R][KV_MAX] softcore LJ at each distinct lambda_v
    long long* ukn_c;              // [R][2] unit-scaled ligand-env / ligand-ligand Coulomb
    // schedules (per schedule id)
    const dbl4* sched_state;      // [MAX_SCHED][K_MAX] lambda_r, lambda_q, lambda_v, kv index
    const int* sched_K;            // [MAX_SCHED]
    const float* kv_lam;           // [MAX_SCHED][KV_MAX] distinct lambda_v values
    const float* kv_A;             // [MAX_SCHED][KV_MAX] alpha (1 - lambda)^p
    const double* kv_dlam;         // FP64 copies
    const double* kv_dA;
    double* out_energy;            // [R][ABFE_N_ENERGY]
    double* out_dudl;              // [R][ABFE_N_DUDL]
    double* out_ukn;               // [R][ukn_ld]
    double* out_du;                // [R][ukn_ld]
    int ukn_ld;
    long long* pair_cnt;           // [R][2] pair counting mode
    int* atom_cnt;                 // [S] per-slot partner counts (counting mode)
    Counters* cnt;
    const StepParams* sp;
    // parameters
    float rc2, rlist;              // r_c^2, outer list radius r_c + skin
    float rin2;                    // (r_c + prune_skin + slack)^2: inner list radius
    float skin_out_half2;          // rebuild when the max squared displacement from
                                   // the build positions > (skin / 2)^2
    float skin_in_half2;           // re-prune a replica when the largest squared
                                   // displacement of its atoms from its prune
                                   // positions > (prune_skin / 2)^2
    float beta, pbeta, nb2l2e, tbsp, sqrt_ke;
    const float4* ewtab;           // [EW_NT] Coulomb force table (see ewald_table)
    int pme;                       // 1 = reciprocal-space Ewald terms are on
    const double2* pme_self;       // [systems] self energy of the environment / ligand charges
    float ewtab_inv_h;             // grid points per unit of r (nm^-1)
    double drc2, dbeta, dke;
    int group, max_entries, ligand_mode;
    int ex_every;                  // steps between in-loop exchange attempts (0 = none)
    unsigned long long ex_seed;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ float rsqrt_fast(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// erfc(t) * exp(t^2) for 0 <= t <= 3.6 from the library's own fit (see
// erfc_coeffs.h). Estrin's scheme: dependency depth 4 instead of Horner's 8
// (binary32 error 4.2e-7 max relative on [0, 3.3], as Horner's 3.9e-7).
__device__ __forceinline__ float erfcx_fit(float t) {
    const float u = rcp_fast(fmaf(ABFE_ERFC_PSUB, t, 1.0f));
    const float u2 = u * u, u4 = u2 * u2;
    const float p01 = fmaf(ABFE_ERFC_Q1, u, ABFE_ERFC_Q0);
    const float p23 = fmaf(ABFE_ERFC_Q3, u, ABFE_ERFC_Q2);
    const float p45 = fmaf(ABFE_ERFC_Q5, u, ABFE_ERFC_Q4);
    const float p67 = fmaf(ABFE_ERFC_Q7, u, ABFE_ERFC_Q6);
    const float q = fmaf(fmaf(p67, u2, p45), u4, fmaf(p23, u2, p01));
    return q * u;
}

__device__ __forceinline__ long long to_fixed(float f) {
    return __float2ll_rn(f * FSCALEF);
}
__device__ __forceinline__ long long to_fixed_d(double f) {
    return __double2ll_rn(f * FSCALE);
}
__device__ __forceinline__ void add_fixed(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

// shift of an entry's j cluster, from its packed y word
__device__ __forceinline__ void entry_shift(int y, float bx, float by, float bz, float& sx,
                                            float& sy, float& sz) {
    const int ix = (y >> 8) & 3, iy = (y >> 10) & 3, iz = (y >> 12) & 3;
    sx = ix == 1 ? 0.0f : (ix == 0 ? -bx : bx);
    sy = iy == 1 ? 0.0f : (iy == 0 ? -by : by);
    sz = iz == 1 ? 0.0f : (iz == 0 ? -bz : bz);
}

__device__ __forceinline__ void set_err(Counters* c, int bit, int info0 = 0, int info1 = 0,
                                        int info2 = 0) {
    if ((atomicOr(&c->err, bit) & bit) == 0) {
        c->err_info[0] = info0;
        c->err_info[1] = info1;
        c->err_info[2] = info2;
    }
}

// Element `it` of an iteration space over per-replica regions (pref: the
// [R + 1] prefix of the replicas' counts, base: the regions' first elements):
// the last replica r with pref[r] <= it holds it (an empty replica shares its
// successor's prefix).
__device__ __forceinline__ int region_index(const int* pref, const int* base, int R, int it) {
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pref[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return base[lo] + (it - pref[lo]);
}

// Exclusive prefix over replicas of min(cnt[r], cap[r]) into pref[0..R] by one
// block (all threads call it); returns the total to every thread.
__device__ __forceinline__ int block_prefix(const int* cnt, const int* cap, int* pref, int R) {
    __shared__ int s_w[32];
    __shared__ int s_carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = 0;
    for (int r0 = 0; r0 < R; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        const int v = r < R ? min(cnt[r], cap[r]) : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) s_w[w] = x;
        __syncthreads();
        int before = s_carry;
        for (int k = 0; k < w; ++k) before += s_w[k];
        if (r < R) pref[r] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = before + x;
        __syncthreads();
    }
    const int total = s_carry;
    if (threadIdx.x == 0) pref[R] = total;
    return total;
}

// ---------------------------------------------------------------- launch wrappers
// (defined in the .cu files; all enqueue on the given stream)
void launch_rebuild(const DevPtrs& P, cudaStream_t s, int n_sm);
void launch_list_build(const DevPtrs& P, cudaStream_t s, int max_lig_cl);
void launch_prune(const DevPtrs& P, cudaStream_t s, int n_sm);
void launch_env_forces(const DevPtrs& P, cudaStream_t s, bool energy, int precision, int grid,
                       int block);
int env_kernel_occupancy(int block, int precision, bool energy);
void launch_lig_forces(const DevPtrs& P, cudaStream_t s, int precision, int grid, int block,
                       bool energy);
void launch_lig_ukn(const DevPtrs& P, cudaStream_t s, int grid, int precision);
void launch_count_pairs(const DevPtrs& P, cudaStream_t s, int grid, int block);
void launch_integrate(const DevPtrs& P, cudaStream_t s, int n_sm);
void launch_step_end(const DevPtrs& P, cudaStream_t s, int inc_step, int force_rebuild,
                     int force_prune, cudaGraphConditionalHandle h_rebuild,
                     cudaGraphConditionalHandle h_prune, cudaGraphConditionalHandle h_exchange,
                     int use_handle);
void launch_bonds(const DevPtrs& P, cudaStream_t s, int precision, bool energy);
void launch_torsions(const DevPtrs& P, cudaStream_t s, int max_tors);
// alchemical waters: slot charges at every replica's lambda_q; energy-pass sums
void launch_aw_refresh(const DevPtrs& P, cudaStream_t s);
void launch_aw_sums(const DevPtrs& P, cudaStream_t s, int max_aw);
void launch_boresch(const DevPtrs& P, cudaStream_t s);
void launch_finalize(const DevPtrs& P, cudaStream_t s);
void launch_ukn_assemble(const DevPtrs& P, cudaStream_t s, double kT);
void launch_scatter_out(const DevPtrs& P, cudaStream_t s, int what, double* outd, float* outf,
                        int n_sm);
void launch_gather_in(const DevPtrs& P, cudaStream_t s, int what, const double* in, int n_sm);

// Smooth-PME grids of all replicas (see pme.cu).
constexpr int PME_KMAX = 256;     // largest grid dimension
constexpr int PME_FFT_LINES = 16;  // neighbouring grid lines per FFT tile (one thread block)
struct PmeDev {
    int R, order;
    const int4* dims;             // [R] K1, K2, K3, -
    const long long* goff;        // [R+1] first grid point of each replica
    int kmax;                     // longest grid line of all replicas
    const int* tiles[3];          // [R+1] per FFT axis: prefix of PME_FFT_LINES-line tiles
    int n_tiles[3];
    const int* tile_rep[3];       // [n_tiles[axis]] replica of each FFT tile
    const int* chunks;            // [R+1] prefix of 256-point chunks of the grids
    const int* chunk_rep;         // [n_chunks] replica of each chunk
    int n_chunks;
    long long total;              // grid points of all replicas
    const double* infl;           // per system: B(m) C(m) at every grid point (0 at m = 0)
    const long long* infl_off;    // [systems]
    const float2* twf;            // exp(-2 pi i k / n) for every FFT length n in use (FP32)
    const double2* twd;           // the same in FP64
    const int* tw_off;            // [PME_KMAX + 1] offset of length n's table (-1: unused)
    long long* qgrid;             // [total] fixed-point charge grid (2^40 units)
    float2* cgrid;                // [total] complex FP32 grid
    double2* dgrid;               // [total] complex FP64 grid (energy split on export passes)
    double beta;
};
// shared-memory attributes of the FFT kernels, sized for the longest line any
// context may use (PME_KMAX; a per-process setting), and a check of M.kmax (host only)
cudaError_t pme_prepare(PmeDev& M);
void launch_pme_forces(const DevPtrs& P, const PmeDev& M, cudaStream_t s, int n_sm, bool energy);
void launch_pme_decomposition(const DevPtrs& P, const PmeDev& M, cudaStream_t s, int n_sm);

// Replica exchange tables. Exchange group = the replicas that share a system and
// a schedule; within a group, positions 0..n-1 list its replicas by ascending
// state (held[] = those states, invariant under exchange: swaps move states
// between replicas, never change the set).
struct ExchangeDev {
    int R;
    const int* grp;        // [R] group of position p
    const int* goff;       // [G+1] first position of each group
    int* slot_rep;         // [R] replica holding the state at position p
    const int* held;       // [R] state index at position p
    int* n_acc;            // accepted swaps of the last attempt
    const double2* sc;     // [MAX_SCHED][K_MAX] softcore alpha (1-lambda_v)^p and its derivative
};
// one attempt (number Counters::ex_attempt) on the given rows, then the attempt
// and acceptance counters advance
void launch_exchange(const DevPtrs& P, RepDev* reps, const ExchangeDev& X, const double* ukn, int ld,
                     unsigned long long seed, cudaStream_t s);

// device memory through the installed allocator hook (else cudaMalloc), for
// entry points without a context; the error string of such calls
void* lib_alloc(size_t bytes, cudaStream_t s);
void lib_free(void* p, size_t bytes, cudaStream_t s);
void set_free_error(const char* msg);

}  // namespace abfe
