// Cell (column) list and cluster-pair list construction for all replicas.
//
// Rebuild pipeline, each stage one kernel over every replica at once:
//   1. k_rb_prepare  (per slot)    copy the slot state aside, wrap positions into
//                                  the box, bin each atom into a z-column (ligand
//                                  atoms into the replica's ligand column);
//   2. k_rb_colscan  (per replica) exclusive scans of the column counts into atom
//                                  and cluster offsets, capacity checks;
//   3. k_rb_fill     (per slot)    scatter old-slot indices into their columns;
//   4. k_rb_sort     (per column)  sort each column by (z, atom index) - the index
//                                  makes the order independent of the scatter -
//                                  and cut it into clusters of 8;
//   5. k_rb_gather   (per slot)    move positions, velocities and parameters into
//                                  the new order (coalesced float4 traffic), write
//                                  the cluster bounding boxes;
//   6. k_build_list  (per i-group) cluster-pair entries within r_c + skin with
//                                  periodic shifts, the cyclic half-list rule,
//                                  exclusion and self-triangle masks, chunked
//                                  work items (cluster-level tests only: the
//                                  prune tests the atoms).
// Every stage first checks Counters::rebuild, so the sequence can also run
// predicated inside a captured step graph.
//
// Prune (k_prune_prep, k_prune; checks Counters::prune): from the outer list,
// at the current positions, the inner list of j rows - per i-cluster the j
// atoms with at least one i atom inside r_c + prune_skin - that the
// environment pair kernel walks until the next prune. Rows with i atoms in
// range in only one half of the cluster follow the full rows (see RowItem).
#include <cuda_runtime.h>

#include <algorithm>

#include "abfe_internal.cuh"

namespace abfe {

namespace {

__device__ __forceinline__ int floor_div(int a, int b) {
    return (a >= 0) ? a / b : -((-a + b - 1) / b);
}

__device__ __forceinline__ float wrapf(float x, float L) {
    float y = x - L * floorf(x / L);
    return (y >= L) ? y - L : y;
}

__global__ void k_rb_prepare(DevPtrs P) {
    if (!P.cnt->rebuild) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.cnt->n_rebuilds += 1;
        P.cnt->build_next = 0;
    }
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        // only the replicas rebuilt in this step (their slots are their own)
        const int rr = P.rep_of_cl[s >> 3];
        if (rr < 0 || !P.bflag[rr]) continue;
        P.perm[s] = -1;
        const int o = P.orig[s];
        float4 x = P.xq[s];
        P.v_old[s] = P.v[s];
        P.orig_old[s] = o;
        if (o < 0) {
            P.xq_old[s] = x;
            continue;
        }
        const int r = P.rep_of_cl[s >> 3];
        const RepDev& R = P.reps[r];
        x.x = wrapf(x.x, R.box[0]);
        x.y = wrapf(x.y, R.box[1]);
        x.z = wrapf(x.z, R.box[2]);
        P.xq_old[s] = x;
        int col;
        if (P.sys_lig[R.sys_atom_off + o]) {
            col = R.ncx * R.ncy;
        } else {
            int ix = (int)(x.x * R.colw_inv[0]);
            int iy = (int)(x.y * R.colw_inv[1]);
            ix = min(max(ix, 0), R.ncx - 1);
            iy = min(max(iy, 0), R.ncy - 1);
            col = ix * R.ncy + iy;
        }
        col += R.col_off;
        P.slot_col[s] = col;
        atomicAdd(&P.col_cnt[col], 1);
    }
}

// One block per replica: exclusive scans over its columns.
__global__ void k_rb_colscan(DevPtrs P) {
    if (!P.cnt->rebuild) return;
    const int r = blockIdx.x;
    if (!P.bflag[r]) return;
    const RepDev R = P.reps[r];
    const int ncol = R.ncx * R.ncy + 1;
    __shared__ int s_warp_a[32], s_warp_c[32];
    __shared__ int s_base_a, s_base_c;
    if (threadIdx.x == 0) { s_base_a = 0; s_base_c = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < ncol; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const int n = (c < ncol) ? P.col_cnt[R.col_off + c] : 0;
        const int ncl = (n + CL - 1) / CL;
        int ia = n, ic = ncl;
        for (int o = 1; o < 32; o <<= 1) {
            const int ta = __shfl_up_sync(0xffffffffu, ia, o);
            const int tc = __shfl_up_sync(0xffffffffu, ic, o);
            if (lane >= o) { ia += ta; ic += tc; }
        }
        if (lane == 31) { s_warp_a[wid] = ia; s_warp_c[wid] = ic; }
        __syncthreads();
        if (wid == 0) {
            int wa = (lane < nw) ? s_warp_a[lane] : 0, wc = (lane < nw) ? s_warp_c[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int ta = __shfl_up_sync(0xffffffffu, wa, o);
                const int tc = __shfl_up_sync(0xffffffffu, wc, o);
                if (lane >= o) { wa += ta; wc += tc; }
            }
            if (lane < nw) { s_warp_a[lane] = wa; s_warp_c[lane] = wc; }
        }
        __syncthreads();
        const int pre_a = s_base_a + (wid ? s_warp_a[wid - 1] : 0) + ia - n;
        const int pre_c = s_base_c + (wid ? s_warp_c[wid - 1] : 0) + ic - ncl;
        if (c < ncol) {
            const int g = R.col_off + c;
            if (n > COL_MAX) set_err(P.cnt, ERRB_COLUMN, g);
            P.col_start[g] = R.cl_off * CL + pre_a;
            P.col_fill[g] = R.cl_off * CL + pre_a;
            P.col_cl_start[g] = R.cl_off + pre_c;
            P.col_ncl[g] = ncl;
            P.col_cnt[g] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_base_a += s_warp_a[nw - 1];
            s_base_c += s_warp_c[nw - 1];
        }
        __syncthreads();
    }
    const int used = s_base_c;
    if (used > R.n_cl_cap) {
        if (threadIdx.x == 0) set_err(P.cnt, ERRB_CLUSTERS, r);
    }
    // clusters beyond the used range hold no atoms in this build
    for (int c = used + threadIdx.x; c < R.n_cl_cap; c += blockDim.x) P.cl_col[R.cl_off + c] = -1;
}

__global__ void k_rb_fill(DevPtrs P) {
    if (!P.cnt->rebuild) return;
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        const int rr = P.rep_of_cl[s >> 3];
        if (rr < 0 || !P.bflag[rr] || P.orig_old[s] < 0) continue;
        const int pos = atomicAdd(&P.col_fill[P.slot_col[s]], 1);
        P.col_atoms[pos] = s;
    }
}

// One warp per column: bitonic sort of (z bits << 32 | atom index) in shared memory.
constexpr int SORT_WARPS = 4;
__global__ void __launch_bounds__(SORT_WARPS * 32) k_rb_sort(DevPtrs P) {
    if (!P.cnt->rebuild) return;
    __shared__ unsigned long long s_key[SORT_WARPS][COL_MAX];
    __shared__ int s_val[SORT_WARPS][COL_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int col = blockIdx.x * SORT_WARPS + w;
    if (col >= P.NCOL) return;
    const int r = P.col_rep[col];
    if (!P.bflag[r]) return;
    const RepDev& R = P.reps[r];
    const bool lig_col = (col - R.col_off) == R.ncx * R.ncy;
    const int start = P.col_start[col];
    int n = P.col_fill[col] - start;
    if (n > COL_MAX) n = COL_MAX;  // error already flagged by the scan
    int np2 = 1;
    while (np2 < n) np2 <<= 1;
    unsigned long long* key = s_key[w];
    int* val = s_val[w];
    for (int k = lane; k < np2; k += 32) {
        if (k < n) {
            const int s = P.col_atoms[start + k];
            const unsigned int o = (unsigned int)P.orig_old[s];
            const unsigned int zb = lig_col ? 0u : __float_as_uint(P.xq_old[s].z);
            key[k] = ((unsigned long long)zb << 32) | o;
            val[k] = s;
        } else {
            key[k] = ~0ull;
            val[k] = -1;
        }
    }
    __syncwarp();
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = lane; k < np2; k += 32) {
                const int partner = k ^ stride;
                if (partner > k) {
                    const bool up = (k & size) == 0;
                    const unsigned long long a = key[k], b = key[partner];
                    if ((a > b) == up) {
                        key[k] = b; key[partner] = a;
                        const int t = val[k]; val[k] = val[partner]; val[partner] = t;
                    }
                }
            }
            __syncwarp();
        }
    }
    const int cl0 = P.col_cl_start[col];
    const int ncl = min(P.col_ncl[col], COL_MAX / CL);
    // a replica whose clusters overflowed its capacity was flagged by the scan;
    // never write outside its own cluster range
    if (cl0 + ncl > R.cl_off + R.n_cl_cap) return;
    for (int k = lane; k < ncl * CL; k += 32) P.perm[cl0 * CL + k] = (k < n) ? val[k] : -1;
    for (int k = lane; k < ncl; k += 32) P.cl_col[cl0 + k] = col;
}

// Per new slot: gather the moved state; 8 consecutive lanes form one cluster
// and reduce its bounding box with width-8 shuffles.
__global__ void k_rb_gather(DevPtrs P) {
    if (!P.cnt->rebuild) return;
    const int lane = threadIdx.x & 31;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int base = warp_global * 32; base < P.S; base += nwarps * 32) {
        const int s = base + lane;
        // slots of the rebuilt replicas (and the padding beyond all replicas)
        const int rs = s < P.S ? P.rep_of_cl[s >> 3] : 0;
        const bool active = s < P.S && (rs < 0 || P.bflag[rs]);
        float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
        if (active) {
            const int old = rs < 0 ? -1 : P.perm[s];
            const int r = P.rep_of_cl[s >> 3];
            if (old < 0 || r < 0) {
                const float4 far = make_float4(DUMMY_FAR + 37.0f * (float)(s & 1023),
                                               DUMMY_FAR + 41.0f * (float)((s >> 10) & 1023),
                                               DUMMY_FAR + 43.0f * (float)((s >> 20) & 1023),
                                               0.0f);
                P.xq[s] = far;
                P.xref[s] = far;
                P.xbuild[s] = far;
                P.v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
                P.se[s] = make_float2(0.f, 0.f);
                P.orig[s] = -1;
            } else {
                const RepDev& R = P.reps[r];
                const int o = P.orig_old[old];
                const float4 prm = P.sys_prm[R.sys_atom_off + o];
                float4 x = P.xq_old[old];
                // alchemical oxygens carry q0 + (1 - lambda_q) dq (0 offset for other atoms)
                x.w = fmaf(1.0f - R.lam_q, P.sys_dq[R.sys_atom_off + o], prm.x);
                P.xq[s] = x;
                P.xref[s] = x;
                P.xbuild[s] = x;
                float4 vv = P.v_old[old];
                vv.w = prm.w;
                P.v[s] = vv;
                P.se[s] = make_float2(prm.y, prm.z);
                P.orig[s] = o;
                P.slot_of[R.atom_off + o] = s;
                lo[0] = hi[0] = x.x;
                lo[1] = hi[1] = x.y;
                lo[2] = hi[2] = x.z;
            }
            P.fx[s] = 0; P.fy[s] = 0; P.fz[s] = 0;
        }
        // ligand clusters (chain order, not spatial) are made whole: every atom
        // takes the image nearest to the cluster's first atom
        {
            const int c = s >> 3;
            const int r = (s < P.S) ? P.rep_of_cl[c] : -1;
            bool ligc = false;
            float box[3] = {1.f, 1.f, 1.f};
            if (r >= 0) {
                const RepDev& R = P.reps[r];
                ligc = P.cl_col[c] == R.col_off + R.ncx * R.ncy;
                box[0] = R.box[0]; box[1] = R.box[1]; box[2] = R.box[2];
            }
            const int leader = lane & ~7;
            float ref[3];
            for (int d = 0; d < 3; ++d) ref[d] = __shfl_sync(0xffffffffu, lo[d], leader);
            if (active && ligc && lo[0] <= hi[0]) {
                float4 x = P.xq[s];
                float* xp[3] = {&x.x, &x.y, &x.z};
                for (int d = 0; d < 3; ++d) {
                    const float dd = *xp[d] - ref[d];
                    *xp[d] = ref[d] + (dd - box[d] * rintf(dd / box[d]));
                    lo[d] = hi[d] = *xp[d];
                }
                P.xq[s] = x;
                P.xref[s] = x;
                P.xbuild[s] = x;
            }
        }
        for (int o = 1; o < 8; o <<= 1) {
            for (int d = 0; d < 3; ++d) {
                lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
        }
        if (active && (lane & 7) == 0) {
            const int c = s >> 3;
            P.clz[c] = make_float2(lo[2], hi[2]);
            if (lo[0] > hi[0]) {
                P.bbc[c] = make_float4(0.f, 0.f, 0.f, -1.f);
                P.bbh[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                P.bbc[c] = make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]),
                                       0.5f * (lo[2] + hi[2]), 1.f);
                P.bbh[c] = make_float4(0.5f * (hi[0] - lo[0]), 0.5f * (hi[1] - lo[1]),
                                       0.5f * (hi[2] - lo[2]), 0.f);
            }
        }
    }
}

// ------------------------------------------------------------------ pair list
//
// One warp builds the list of one i-group. Candidate j clusters are gathered in
// a flattened index space: a warp pass collects the columns within reach of
// the group (slab test) with their cluster ranges and a prefix sum of their
// cluster counts; each lane then takes flat candidate indices, loads the
// candidate's bounding box once (independent, coalesced loads) and tests all
// three z images in registers. Accepted entries go to per-warp shared memory
// with a small hash (j cluster -> chain of entries) used to attach exclusion
// and self-triangle masks; the finished list is appended to the global arrays.
// Both half tiles of an accepted (entry, i-cluster) are marked live: the
// prune decides per atom which rows the pair kernel walks (an atom-level
// half-tile test here took a third of the build time and saved the prune
// less than that).

constexpr int MAXCOL = 96;    // z segments gathered per batch (32 columns x 3 images)
constexpr float ZSLACK = 1e-4f;  // nm: z prefilter margin, far above rounding of the z bounds
constexpr unsigned long long TRI_MASK = 0xFF7F3F1F0F070301ull;  // bits (i, j) with j <= i

template <int ECAP, int HCAP, int XCAP, int GM>
struct LBS {
    int ej[ECAP];             // j cluster
    int ey[ECAP];             // packed y word
    int enext[ECAP];          // next entry with the same j cluster
    int exs[ECAP];            // exclusion slot of the entry or -1
    int hkey[HCAP];
    int hhead[HCAP];
    unsigned long long xm[XCAP][GM];
    int col_cs[MAXCOL], col_pref[MAXCOL + 1], col_k[MAXCOL];
    int n_e, n_x, overflow, n_col;
};

template <int HCAP>
__device__ __forceinline__ unsigned int hash_of(int jc) {
    return ((unsigned int)jc * 2654435761u) >> (32 - __builtin_ctz(HCAP));
}

template <class L_t, int HCAP>
__device__ __forceinline__ void lb_insert(L_t& L, int jc, int e) {
    unsigned int h = hash_of<HCAP>(jc);
    for (int probe = 0; probe < HCAP; ++probe) {
        const int old = atomicCAS(&L.hkey[h], -1, jc);
        if (old == -1 || old == jc) {
            L.enext[e] = atomicExch(&L.hhead[h], e);
            return;
        }
        h = (h + 1) & (HCAP - 1);
    }
    L.overflow = 2;
}

template <class L_t, int HCAP>
__device__ __forceinline__ int lb_find(const L_t& L, int jc) {
    unsigned int h = hash_of<HCAP>(jc);
    for (int probe = 0; probe < HCAP; ++probe) {
        const int k = L.hkey[h];
        if (k == jc) return L.hhead[h];
        if (k == -1) return -1;
        h = (h + 1) & (HCAP - 1);
    }
    return -1;
}

// squared distance between two boxes (centre/half extent) with the second shifted
__device__ __forceinline__ float bb_dist2(float4 c1, float4 h1, float cx, float cy, float cz,
                                          float4 h2) {
    const float dx = fmaxf(fabsf(c1.x - cx) - h1.x - h2.x, 0.f);
    const float dy = fmaxf(fabsf(c1.y - cy) - h1.y - h2.y, 0.f);
    const float dz = fmaxf(fabsf(c1.z - cz) - h1.z - h2.z, 0.f);
    return dx * dx + dy * dy + dz * dz;
}

// Half-list rule: which of the two orderings (ic, jc) / (jc, ic) of a cluster
// pair carries it. With n_wrap > 0 the owner is ic when jc lies in the half of
// the cyclic index range [1, n_wrap/2) after ic (ties at exactly n_wrap/2 go to
// the smaller index): every cluster keeps about half of its neighbours, also at
// the periodic seam of the column order, where the plain rule jc > ic gives the
// first columns full lists and the last ones none. n_wrap = 0 is the plain rule.
// A cluster against its own images keeps one of each +-shift pair and the
// unshifted self image (code 13, masked to its upper triangle later).
__device__ __forceinline__ bool half_owner(int ic, int jc, int code, int n_wrap) {
    if (jc == ic) return code >= 13;
    if (n_wrap <= 0) return jc > ic;
    int d = jc - ic;
    if (d < 0) d += n_wrap;
    return 2 * d < n_wrap || (2 * d == n_wrap && jc > ic);
}

// i-cluster mask of one candidate (j cluster with a loaded box, one image);
// n_wrap < 0: no half-list rule (clusters of different kinds)
template <int G>
__device__ __forceinline__ int lb_mask(const RepDev& R, int c0, int ng, const float4* bc,
                                       const float4* bh, int jc, float4 jb, float4 jh, int sx,
                                       int sy, int sz, int n_wrap, float rl2) {
    int mask = 0;
    const float cx = jb.x + sx * R.box[0], cy = jb.y + sy * R.box[1], cz = jb.z + sz * R.box[2];
    const int code = (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g < ng && bb_dist2(bc[g], bh[g], cx, cy, cz, jh) < rl2) {
            if (n_wrap < 0 || half_owner(c0 + g, jc, code, n_wrap)) mask |= 1 << g;
        }
    }
    return mask;
}

// append accepted candidates (warp-collective; order = lane order)
template <class L_t, int ECAP, int HCAP>
__device__ __forceinline__ void lb_accept(L_t& L, int mask, int jc, int sx, int sy, int sz,
                                          int jlig) {
    const unsigned int ball = __ballot_sync(0xffffffffu, mask != 0);
    if (ball == 0u) return;
    const int lane = threadIdx.x & 31;
    const int base = L.n_e;
    const int pos = base + __popc(ball & ((1u << lane) - 1u));
    const bool ok = mask != 0 && pos < ECAP;
    if (ok) {
        L.ej[pos] = jc;
        L.ey[pos] = pack_entry_y(mask, sx, sy, sz, jlig);
        L.exs[pos] = -1;
    } else if (mask != 0) {
        L.overflow = 1;
    }
    __syncwarp();
    if (ok) lb_insert<L_t, HCAP>(L, jc, pos);
    __syncwarp();
    if (lane == 0) L.n_e = min(base + __popc(ball), ECAP);
    __syncwarp();
}

// Masks, write-out and work items of the entries now in the warp's buffer, then
// an empty buffer. A group whose candidates do not fit into one buffer is
// flushed several times: every (j cluster, image) entry lives in exactly one
// flush, and its exclusion and self-triangle bits are set in that flush.
template <int G, int ECAP, int HCAP, int XCAP, int GM>
__device__ __noinline__ void lb_flush(const DevPtrs& P, LBS<ECAP, HCAP, XCAP, GM>& L, int c, int ng, int r,
                         const RepDev& R, bool is_lig) {
    using L_t = LBS<ECAP, HCAP, XCAP, GM>;
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const int n_e = L.n_e;
    // ---- entries needing masks: excluded partners and the self triangle
    const int sysoff = R.sys_ex_off;
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0 flags entries (exs = -2), pass 1 sets mask bits
        const int a_local = lane;
        if (a_local < ng * CL) {
            const int g = a_local >> 3, ii = a_local & 7;
            const int a = c * CL + a_local;
            const int o = P.orig[a];
            if (o >= 0) {
                const int kb = P.sys_ex_off[sysoff + o], ke = P.sys_ex_off[sysoff + o + 1];
                for (int kk = kb; kk < ke; ++kk) {
                    const int pslot = P.slot_of[R.atom_off + P.sys_ex_idx[kk]];
                    const int jc = pslot >> 3, jl = pslot & 7;
                    for (int e = lb_find<L_t, HCAP>(L, jc); e >= 0; e = L.enext[e]) {
                        if (!entry_g(L.ey[e], g)) continue;
                        if (pass == 0) {
                            L.exs[e] = -2;
                        } else {
                            const int xs = L.exs[e];
                            if (xs >= 0) atomicOr(&L.xm[xs][g], 1ull << (ii * 8 + jl));
                        }
                    }
                }
            }
        }
        for (int e = lane; e < n_e; e += 32) {
            const int jc = L.ej[e];
            const int y = L.ey[e];
            const int g = jc - c;
            if (g >= 0 && g < ng && (y & ENTRY_SHIFT_BITS) == ENTRY_NOSHIFT && entry_g(y, g)) {
                if (pass == 0) L.exs[e] = -2;
                else if (L.exs[e] >= 0) atomicOr(&L.xm[L.exs[e]][g], TRI_MASK);
            }
        }
        __syncwarp();
        if (pass == 0) {
            for (int e0 = 0; e0 < n_e; e0 += 32) {
                const int e = e0 + lane;
                const bool need = (e < n_e) && L.exs[e] == -2;
                const unsigned int b = __ballot_sync(0xffffffffu, need);
                const int pos = L.n_x + __popc(b & ((1u << lane) - 1u));
                if (need) {
                    if (pos < XCAP) {
                        L.exs[e] = pos;
                        for (int gg = 0; gg < GM; ++gg) L.xm[pos][gg] = 0ull;
                    } else {
                        L.exs[e] = -1;
                        L.overflow = 3;
                    }
                }
                __syncwarp();
                if (lane == 0) L.n_x = min(L.n_x + __popc(b), XCAP);
                __syncwarp();
            }
        }
        __syncwarp();
    }
    if (L.overflow) {
        // reason: 1 too many j entries, 2 hash full, 3 too many masked entries
        if (lane == 0) set_err(P.cnt, ERRB_GROUP, c, L.overflow, L.n_e);
        return;
    }
    // ---- write out (masked entries keep their place in the masked list)
    const int n_x = L.n_x;
    int n_plain = 0;
    for (int e0 = 0; e0 < n_e; e0 += 32) {
        const int e = e0 + lane;
        n_plain += __popc(__ballot_sync(0xffffffffu,
                                        (e < n_e) && L.exs[e] < 0 && (L.ey[e] & 0xFF) != 0));
    }
    // offsets in this replica's regions
    int e_base = 0, x_base = 0;
    if (lane == 0) {
        e_base = atomicAdd(&P.n_entries_r[r], n_plain);
        x_base = atomicAdd(&P.n_xentries_r[r], n_x);
    }
    e_base = __shfl_sync(0xffffffffu, e_base, 0);
    x_base = __shfl_sync(0xffffffffu, x_base, 0);
    if (e_base + n_plain > P.ent_cap[r] || x_base + n_x > P.xent_cap[r]) {
        if (lane == 0) {
            const bool xe = x_base + n_x > P.xent_cap[r];
            set_err(P.cnt, ERRB_LIST, c, (r << 4) | (xe ? OVF_XENTRIES : OVF_ENTRIES),
                    xe ? x_base + n_x : e_base + n_plain);
        }
        return;
    }
    e_base += P.ent_base[r];
    x_base += P.xent_base[r];
    int written = 0;
    for (int e0 = 0; e0 < n_e; e0 += 32) {
        const int e = e0 + lane;
        const bool plain = (e < n_e) && L.exs[e] < 0 && (L.ey[e] & 0xFF) != 0;
        const unsigned int b = __ballot_sync(0xffffffffu, plain);
        if (plain) {
            P.entries[e_base + written + __popc(b & ((1u << lane) - 1u))] =
                make_int2(L.ej[e], L.ey[e]);
        } else if (e < n_e && L.exs[e] >= 0) {
            const int xs = L.exs[e];
            P.xentries[x_base + xs] = make_int2(L.ej[e], L.ey[e]);
            for (int gg = 0; gg < GMAX; ++gg)
                P.xmasks[(size_t)(x_base + xs) * GMAX + gg] = gg < GM ? L.xm[xs][gg] : 0ull;
        }
        written += __popc(b);
    }
    if (n_plain + n_x == 0) return;
    const int chunk = is_lig ? min(P.max_entries, 16) : P.max_entries;
    const int n_items = max(1, (n_plain + chunk - 1) / chunk);
    int ib = 0;
    if (lane == 0) ib = atomicAdd(is_lig ? &P.n_items_lig_r[r] : &P.n_items_env_r[r], n_items);
    ib = __shfl_sync(0xffffffffu, ib, 0);
    const int cap = is_lig ? P.ilig_cap[r] : P.ienv_cap[r];
    if (ib + n_items > cap) {
        if (lane == 0)
            set_err(P.cnt, ERRB_LIST, c, (r << 4) | (is_lig ? OVF_ITEMS_LIG : OVF_ITEMS_ENV),
                    ib + n_items);
        return;
    }
    ib += is_lig ? P.ilig_base[r] : P.ienv_base[r];
    Item* items = is_lig ? P.items_lig : P.items_env;
    for (int t = lane; t < n_items; t += 32) {
        Item it;
        it.c0 = c;
        it.ng = ng;
        it.rep = r;
        it.e_begin = e_base + t * chunk;
        it.e_cnt = max(0, min(chunk, n_plain - t * chunk));
        it.x_begin = x_base;
        it.x_cnt = (t == 0) ? n_x : 0;
        it.flags = 0;
        items[ib + t] = it;
    }
}

template <class L_t, int HCAP>
__device__ __forceinline__ void lb_reset(L_t& L) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    for (int h = lane; h < HCAP; h += 32) { L.hkey[h] = -1; L.hhead[h] = -1; }
    if (lane == 0) { L.n_e = 0; L.n_x = 0; L.overflow = 0; }
    __syncwarp();
}

// Clusters of one column (n clusters sorted by z, z bounds zb[k] = (min, max))
// whose z extent overlaps [wlo, whi]: the index range [a, b). Starts from the
// index a uniform column would give and walks to the exact bounds; the bounds
// are monotonic in k because the column is sorted by z.
__device__ __forceinline__ void z_range(const float2* zb, int n, float wlo, float whi,
                                        float invLz, int& a_out, int& b_out) {
    int a = min(max((int)(wlo * invLz * n) - 1, 0), n);
    while (a > 0 && zb[a - 1].y >= wlo) --a;
    while (a < n && zb[a].y < wlo) ++a;
    int b = min(max((int)(whi * invLz * n) + 2, a), n);
    while (b < n && zb[b].x <= whi) ++b;
    while (b > a && zb[b - 1].x > whi) --b;
    a_out = a;
    b_out = b;
}

template <int G, int ECAP, int HCAP, int XCAP, int GM>
__device__ void build_group(const DevPtrs& P, LBS<ECAP, HCAP, XCAP, GM>& L, int c, bool is_lig) {
    using L_t = LBS<ECAP, HCAP, XCAP, GM>;
    const int lane = threadIdx.x & 31;
    const int col = P.cl_col[c];
    const int r = P.rep_of_cl[c];
    const RepDev R = P.reps[r];
    const int lig_col = R.col_off + R.ncx * R.ncy;
    // environment clusters of the replica: [R.cl_off, start of the ligand column)
    const int n_env = P.col_cl_start[lig_col] - R.cl_off;
    const int k = c - P.col_cl_start[col];
    const int ng = is_lig ? 1 : min(G, P.col_ncl[col] - k);

    float4 bc[G], bh[G];
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g < ng) {
            bc[g] = P.bbc[c + g];
            bh[g] = P.bbh[c + g];
            if (bc[g].w > 0.f) {
                lo[0] = fminf(lo[0], bc[g].x - bh[g].x); hi[0] = fmaxf(hi[0], bc[g].x + bh[g].x);
                lo[1] = fminf(lo[1], bc[g].y - bh[g].y); hi[1] = fmaxf(hi[1], bc[g].y + bh[g].y);
                lo[2] = fminf(lo[2], bc[g].z - bh[g].z); hi[2] = fmaxf(hi[2], bc[g].z + bh[g].z);
            }
        } else {
            bc[g] = make_float4(0.f, 0.f, 0.f, -1.f);
            bh[g] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    lb_reset<L_t, HCAP>(L);
    const float rl = P.rlist, rl2 = rl * rl;
    if (lo[0] <= hi[0]) {
        const int ixlo = (int)floorf((lo[0] - rl) * R.colw_inv[0]);
        const int ixhi = (int)floorf((hi[0] + rl) * R.colw_inv[0]);
        const int iylo = (int)floorf((lo[1] - rl) * R.colw_inv[1]);
        const int iyhi = (int)floorf((hi[1] + rl) * R.colw_inv[1]);
        const int nyr = iyhi - iylo + 1;
        const int ncand = (ixhi - ixlo + 1) * nyr;
        const float cwx = R.box[0] / R.ncx, cwy = R.box[1] / R.ncy;
        const float zlo = lo[2] - rl - ZSLACK, zhi = hi[2] + rl + ZSLACK;
        const float Lz = R.box[2], invLz = 1.0f / R.box[2];
        for (int cb = 0; cb < ncand; cb += 32) {
            // (a) segments of this batch of 32 columns: for each column that the
            // group can reach in x/y and each z image, the range of its clusters
            // (sorted by z) whose z extent overlaps the group's z window
            if (lane == 0) L.n_col = 0;
            __syncwarp();
            {
                const int q = cb + lane;
                bool ok = q < ncand;
                int kx = 0, ky = 0, jcol = 0;
                if (ok) {
                    const int ix = ixlo + q / nyr, iy = iylo + q % nyr;
                    kx = floor_div(ix, R.ncx);
                    ky = floor_div(iy, R.ncy);
                    const int wx = ix - kx * R.ncx, wy = iy - ky * R.ncy;
                    // (1e-5 nm of slack keeps this coarse test more inclusive than the
                    // exact bounding-box test under rounding)
                    const float dxc = fmaxf(fmaxf(ix * cwx - hi[0], lo[0] - (ix + 1) * cwx) - 1e-5f, 0.f);
                    const float dyc = fmaxf(fmaxf(iy * cwy - hi[1], lo[1] - (iy + 1) * cwy) - 1e-5f, 0.f);
                    ok = kx >= -1 && kx <= 1 && ky >= -1 && ky <= 1 && dxc * dxc + dyc * dyc < rl2;
                    jcol = R.col_off + wx * R.ncy + wy;
                }
                const int cs = ok ? P.col_cl_start[jcol] : 0;
                const int n = ok ? P.col_ncl[jcol] : 0;
#pragma unroll
                for (int kz = -1; kz <= 1; ++kz) {
                    // j clusters of image kz: z_j + kz Lz in [zlo, zhi], z_j in [0, Lz)
                    const float wlo = zlo - kz * Lz, whi = zhi - kz * Lz;
                    int a = 0, b = 0;
                    if (n > 0 && whi >= 0.f && wlo < Lz)
                        z_range(P.clz + cs, n, fmaxf(wlo, 0.f), fminf(whi, Lz), invLz, a, b);
                    const bool has = b > a;
                    const unsigned int bl = __ballot_sync(0xffffffffu, has);
                    if (has) {
                        const int slot = L.n_col + __popc(bl & ((1u << lane) - 1u));
                        L.col_cs[slot] = cs + a;
                        L.col_pref[slot] = b - a;
                        L.col_k[slot] = (kx + 1) | ((ky + 1) << 2) | ((kz + 1) << 4);
                    }
                    __syncwarp();
                    if (lane == 0) L.n_col += __popc(bl);
                    __syncwarp();
                }
            }
            const int ncol = L.n_col;
            // (b) exclusive prefix of the segment lengths (warp scans of 32)
            int carry = 0;
            for (int hlf = 0; hlf < ncol; hlf += 32) {
                const int q = hlf + lane;
                const int v = q < ncol ? L.col_pref[q] : 0;
                int x = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += t;
                }
                __syncwarp();
                if (q < ncol) L.col_pref[q] = carry + x - v;
                carry += __shfl_sync(0xffffffffu, x, 31);
                __syncwarp();
            }
            if (lane == 0) L.col_pref[ncol] = carry;
            __syncwarp();
            const int T = carry;
            // (c) flattened candidates, one image each; the segment lookup and the
            // box loads of the next 32 candidates are issued before the current
            // ones are tested
            auto fetch = [&](int t, int& jc, int& kk, float4& jb, float4& jh) {
                jc = 0; kk = 0x15;  // (0, 0, 0) image
                jb = make_float4(0.f, 0.f, 0.f, -1.f);
                jh = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t < T) {
                    int a = 0, b = ncol - 1;  // last segment with col_pref <= t
                    while (a < b) {
                        const int mid = (a + b + 1) >> 1;
                        if (L.col_pref[mid] <= t) a = mid; else b = mid - 1;
                    }
                    jc = L.col_cs[a] + (t - L.col_pref[a]);
                    kk = L.col_k[a];
                    jb = P.bbc[jc];
                    jh = P.bbh[jc];
                }
            };
            int jc_n, kk_n;
            float4 jb_n, jh_n;
            fetch(lane, jc_n, kk_n, jb_n, jh_n);
            for (int t0 = 0; t0 < T; t0 += 32) {
                const int jc = jc_n, kk = kk_n;
                const float4 jb = jb_n, jh = jh_n;
                if (t0 + 32 < T) fetch(t0 + 32 + lane, jc_n, kk_n, jb_n, jh_n);
                const int kx = (kk & 3) - 1, ky = ((kk >> 2) & 3) - 1, kz = ((kk >> 4) & 3) - 1;
                const int m = jb.w > 0.f ? lb_mask<G>(R, c, ng, bc, bh, jc, jb, jh, kx, ky, kz,
                                                      is_lig ? -1 : n_env, rl2)
                                         : 0;
                // up to 32 accepts follow: flush a buffer that might not hold them
                __syncwarp();
                if (L.n_e > ECAP - 32) {
                    lb_flush<G, ECAP, HCAP, XCAP, GM>(P, L, c, ng, r, R, is_lig);
                    lb_reset<L_t, HCAP>(L);
                }
                lb_accept<L_t, ECAP, HCAP>(L, m, jc, kx, ky, kz, 0);
            }
        }
        // ligand clusters (only for ligand i-clusters; all 27 images)
        if (is_lig) {
            const int cs = P.col_cl_start[lig_col], nc = P.col_ncl[lig_col];
            for (int t0 = 0; t0 < nc * 27; t0 += 32) {
                __syncwarp();
                if (L.n_e > ECAP - 32) {
                    lb_flush<G, ECAP, HCAP, XCAP, GM>(P, L, c, ng, r, R, is_lig);
                    lb_reset<L_t, HCAP>(L);
                }
                const int t = t0 + lane;
                const bool valid = t < nc * 27;
                const int jc = valid ? cs + t / 27 : cs;
                const int code = valid ? t % 27 : 13;
                int m = 0;
                if (valid) {
                    const float4 jb = P.bbc[jc], jh = P.bbh[jc];
                    if (jb.w > 0.f)
                        m = lb_mask<G>(R, c, ng, bc, bh, jc, jb, jh, code % 3 - 1,
                                       (code / 3) % 3 - 1, code / 9 - 1, 0, rl2);
                }
                lb_accept<L_t, ECAP, HCAP>(L, m, jc, code % 3 - 1, (code / 3) % 3 - 1,
                                           code / 9 - 1, 1);
            }
        }
    }
    lb_flush<G, ECAP, HCAP, XCAP, GM>(P, L, c, ng, r, R, is_lig);
}


// environment groups: 256 entries, 256 hash buckets, 64 masked entries per warp
// buffer (a longer list is flushed in parts)
constexpr int ENV_E = 256, ENV_H = 256, ENV_X = 64, ENV_WARPS = 4;
// ligand clusters: no half-list rule against the environment, so larger lists
constexpr int LIG_E = 1024, LIG_H = 1024, LIG_X = 128, LIG_WARPS = 2;

// Persistent: each warp takes chunks of `chunk` consecutive clusters and builds
// the groups that start in them (the first cluster of every G in a column), so
// no warp of a resident block idles on clusters that start no group. The chunk
// (1..32) shrinks for small systems so that every warp gets work. Six blocks
// per SM (registers capped at 80): the few spills cost less than the latency
// the extra warps hide (60.9 vs 66.8 ms per build of the 1,152-window batch
// at the four blocks that 128 registers allow).
template <int G>
__global__ void __launch_bounds__(ENV_WARPS * 32, 6) k_build_list_env(DevPtrs P, int chunk) {
    if (!P.cnt->rebuild) return;
    extern __shared__ unsigned char lb_smem[];
    using L_t = LBS<ENV_E, ENV_H, ENV_X, G>;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    L_t& L = reinterpret_cast<L_t*>(lb_smem)[w];
    for (;;) {
        int c0 = 0;
        if (lane == 0) c0 = atomicAdd(&P.cnt->build_next, chunk);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if (c0 >= P.C) break;
        const int c1 = min(c0 + chunk, P.C);
        for (int c = c0; c < c1; ++c) {
            const int rc = P.rep_of_cl[c];
            if (rc < 0 || !P.bflag[rc]) continue;   // replica keeps its outer list
            const int col = P.cl_col[c];
            if (col < 0) continue;
            const RepDev& R = P.reps[P.rep_of_cl[c]];
            if (col == R.col_off + R.ncx * R.ncy) continue;   // ligand clusters: k_build_list_lig
            if ((c - P.col_cl_start[col]) % G) continue;      // not the first cluster of its group
            build_group<G, ENV_E, ENV_H, ENV_X, G>(P, L, c, false);
        }
    }
}

// one warp per (replica, ligand cluster)
__global__ void __launch_bounds__(LIG_WARPS * 32) k_build_list_lig(DevPtrs P, int max_lig_cl) {
    if (!P.cnt->rebuild) return;
    extern __shared__ unsigned char lb_smem[];
    using L_t = LBS<LIG_E, LIG_H, LIG_X, 1>;
    const int w = threadIdx.x >> 5;
    L_t& L = reinterpret_cast<L_t*>(lb_smem)[w];
    const int gw = blockIdx.x * LIG_WARPS + w;
    const int r = gw / max_lig_cl, k = gw % max_lig_cl;
    if (r >= P.R || !P.bflag[r]) return;
    const RepDev& R = P.reps[r];
    const int lig_col = R.col_off + R.ncx * R.ncy;
    if (k >= P.col_ncl[lig_col]) return;
    build_group<1, LIG_E, LIG_H, LIG_X, 1>(P, L, P.col_cl_start[lig_col] + k, true);
}

// ------------------------------------------------------------------ prune
//
// Exactness: the outer list holds every pair that comes within r_c before the
// next rebuild (no atom moves more than skin/2 from its build position until
// then); a pair that comes within r_c before the next prune is at most
// prune_skin away from r_c at the prune (no atom moves more than prune_skin/2
// from its prune position), so the inner list at r_c + prune_skin holds it.

// Positions of this prune (the displacement reference of the integrator) and
// every cluster's bounding box at these positions (centre, half extent; .w of the
// half extent = the cluster's atom count, its atoms being its first slots;
// centre .w < 0 for an empty cluster). Eight consecutive lanes are one cluster.
__global__ void k_prune_prep(DevPtrs P) {
    if (!P.cnt->prune) return;
    const int lane = threadIdx.x & 31;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int base = warp_global * 32; base < P.S; base += nwarps * 32) {
        const int s = base + lane;
        const int rep = s < P.S ? P.rep_of_cl[s >> 3] : -1;
        const bool active = rep >= 0 && P.pflag[rep];   // replicas pruned in this step
        float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
        int real = 0;
        if (active) {
            const float4 x = P.xq[s];
            P.xref[s] = x;
            if (P.orig[s] >= 0) {
                lo[0] = hi[0] = x.x;
                lo[1] = hi[1] = x.y;
                lo[2] = hi[2] = x.z;
                real = 1;
            }
        }
        for (int o = 1; o < 8; o <<= 1) {
            for (int d = 0; d < 3; ++d) {
                lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
            }
            real += __shfl_xor_sync(0xffffffffu, real, o);
        }
        if (active && (lane & 7) == 0) {
            const int c = s >> 3;
            if (real == 0) {
                P.bbc[c] = make_float4(0.f, 0.f, 0.f, -1.f);
                P.bbh[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                P.bbc[c] = make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]),
                                       0.5f * (lo[2] + hi[2]), 1.f);
                P.bbh[c] = make_float4(0.5f * (hi[0] - lo[0]), 0.5f * (hi[1] - lo[1]),
                                       0.5f * (hi[2] - lo[2]), (float)real);
            }
        }
    }
}

constexpr int PR_WARPS = 4;
constexpr int PR_CHUNK = 16;          // outer items claimed at once by a warp
constexpr int PR_ECAP = 512;          // plain entries per outer work item (max_entries <= 512)
constexpr int PR_XCAP = ENV_X;        // masked entries per outer work item

__device__ __forceinline__ float dist2(const float4& a, float x, float y, float z) {
    const float dx = x - a.x, dy = y - a.y, dz = z - a.z;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// One warp per outer environment work item, in two passes over its entries.
// (a) Lane per entry: with the clusters' bounding boxes at the current
// positions, each (entry, i-cluster) is sorted as "no row" (boxes farther
// apart than the inner radius), "every j atom a row" (farthest points within
// it, both half tiles live, no excluded pair) or "test"; the tests are queued
// in shared memory. (b) Lane per j row, four queued tests per pass (lane = jj +
// 8 e): the lane loads its j atom (eight lanes read the entry's 128-byte line)
// and tests it against all 8 i atoms without branches, in coordinates relative
// to the i-cluster's box centre: r^2 - r_in^2 = |x_j|^2 + (|x_i|^2 - r_in^2 -
// 2 x_j.x_i), three FMAs and a min per i atom; a row is live in a half (i
// atoms 0-3 or 4-7) if the half tile is live and the smallest bracket over
// the half's atoms that are not excluded is below -|x_j|^2. Rows without
// excluded pairs go to the plain row list (full rows, then rows with only
// atoms 0-3, then only atoms 4-7, in range), rows with excluded pairs (masked
// entries only) to the masked row list with their 8-bit mask of excluded i
// atoms. Row order within each run follows the outer entries.
// per-warp prune state (dynamic shared memory)
template <int G>
struct PrS {
    float4 xi[G * CL];     // -2 x_i', |x_i'|^2 - r_in^2 (x_i' = x_i - box centre)
    float4 bb[G][2];       // i-cluster box: centre, half extent
    float4 sh[28];         // image shifts of the item's replica, by code
    unsigned int word[PR_ECAP + PR_XCAP];        // entry's row word for its j atom 0
    unsigned short test[(PR_ECAP + PR_XCAP) * G];  // queued (entry, i-cluster) tests
    // per (entry, i-cluster): bit jj = row jj has an atom of i atoms 0-3 (lo)
    // or of i atoms 4-7 (hi) inside the inner radius
    unsigned char lo[PR_ECAP + PR_XCAP][G];
    unsigned char hi[PR_ECAP + PR_XCAP][G];
    int ntest;
};

template <int G>
__global__ void __launch_bounds__(PR_WARPS * 32) k_prune(DevPtrs P) {
    if (!P.cnt->prune) return;
    extern __shared__ __align__(16) unsigned char pr_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    PrS<G>& S = reinterpret_cast<PrS<G>*>(pr_smem)[w];
    const int n_items = P.ienv_pref[P.R];
    const float rin2 = P.rin2;
    // items are claimed in chunks of PR_CHUNK (a prune of a few windows skips
    // most items: one claim per item would serialise on the counter), and the
    // items of a window that keeps its rows are skipped as a range
    // (fewer at once when there are few items per warp)
    const int chunk = max(1, min(PR_CHUNK, n_items / ((int)gridDim.x * PR_WARPS * 4)));
    int it_next = 0, it_end = 0;
    for (;;) {
        if (it_next >= it_end) {
            int c0 = 0;
            if (lane == 0) c0 = atomicAdd(&P.cnt->prune_next, chunk);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if (c0 >= n_items) break;
            it_next = c0;
            it_end = min(c0 + chunk, n_items);
        }
        const int it = it_next++;
        int rr = 0, hi = P.R - 1;   // the window of item it
        while (rr < hi) {
            const int mid = (rr + hi + 1) >> 1;
            if (P.ienv_pref[mid] <= it) rr = mid;
            else hi = mid - 1;
        }
        if (!P.pflag[rr]) {   // this window keeps its rows
            it_next = min(it_end, P.ienv_pref[rr + 1]);
            continue;
        }
        const Item I = P.items_env[P.ienv_base[rr] + (it - P.ienv_pref[rr])];
        if (I.e_cnt > PR_ECAP || I.x_cnt > PR_XCAP) {
            if (lane == 0)
                set_err(P.cnt, ERRB_LIST, I.c0, (I.rep << 4) | OVF_PRUNE_ITEM,
                        I.e_cnt > PR_ECAP ? I.e_cnt : I.x_cnt);
            continue;
        }
        const RepDev& R = P.reps[I.rep];
        if (lane < G) {
            S.bb[lane][0] = lane < I.ng ? P.bbc[I.c0 + lane] : make_float4(0.f, 0.f, 0.f, -1.f);
            S.bb[lane][1] = lane < I.ng ? P.bbh[I.c0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (lane < 27)
            S.sh[lane] = make_float4((float)(lane % 3 - 1) * R.box[0],
                                     (float)((lane / 3) % 3 - 1) * R.box[1],
                                     (float)(lane / 9 - 1) * R.box[2], 0.f);
        if (lane == 0) S.ntest = 0;
        __syncwarp();
        if (lane < G * CL) {
            const int g = lane >> 3;
            float4 v = make_float4(0.f, 0.f, 0.f, 3.0e30f);   // never inside
            if (g < I.ng) {
                const float4 x = P.xq[(I.c0 + g) * CL + (lane & 7)];
                const float4 c = S.bb[g][0];
                if (fabsf(x.x) < 5.0e3f && c.w > 0.f) {       // a real atom (padding lies far out)
                    const float dx = x.x - c.x, dy = x.y - c.y, dz = x.z - c.z;
                    v = make_float4(-2.f * dx, -2.f * dy, -2.f * dz,
                                    fmaf(dx, dx, fmaf(dy, dy, dz * dz)) - rin2);
                }
            }
            S.xi[lane] = v;
        }
        __syncwarp();
        const int n_e = I.e_cnt + I.x_cnt;
        // (a) box classification, lane per entry
        for (int t0 = 0; t0 < n_e; t0 += 32) {
            const int t = t0 + lane;
            unsigned int need = 0u;   // bit g: test rows of i-cluster g
            if (t < n_e) {
                const bool xm = t >= I.e_cnt;
                const int k = xm ? I.x_begin + (t - I.e_cnt) : I.e_begin + t;
                const int2 e = xm ? P.xentries[k] : P.entries[k];
                float sx, sy, sz;
                entry_shift(e.y, R.box[0], R.box[1], R.box[2], sx, sy, sz);
                const int code = ((e.y >> 8) & 3) + 3 * ((e.y >> 10) & 3) + 9 * ((e.y >> 12) & 3);
                S.word[t] = ((unsigned int)code << ROW_SLOT_BITS) | (unsigned int)(e.x * CL);
                const float4 jb = P.bbc[e.x], jh = P.bbh[e.x];
                const unsigned int all = jb.w > 0.f ? (1u << (int)jh.w) - 1u : 0u;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    unsigned int live = 0u;
                    const float4 ic = S.bb[g][0], ih = S.bb[g][1];
                    if (g < I.ng && entry_g(e.y, g) && all && ic.w > 0.f) {
                        const float ax = fabsf(jb.x + sx - ic.x), ay = fabsf(jb.y + sy - ic.y),
                                    az = fabsf(jb.z + sz - ic.z);
                        const float nx = fmaxf(ax - jh.x - ih.x, 0.f), ny = fmaxf(ay - jh.y - ih.y, 0.f),
                                    nz = fmaxf(az - jh.z - ih.z, 0.f);
                        if (fmaf(nx, nx, fmaf(ny, ny, nz * nz)) < rin2) {
                            const float fx = ax + jh.x + ih.x, fy = ay + jh.y + ih.y,
                                        fz = az + jh.z + ih.z;
                            const bool masked = xm && P.xmasks[(size_t)k * GMAX + g] != 0ull;
                            if (((e.y >> (2 * g)) & 3) == 3 && !masked &&
                                fmaf(fx, fx, fmaf(fy, fy, fz * fz)) < rin2)
                                live = all;            // every pair within the inner radius
                            else
                                need |= 1u << g;
                        }
                    }
                    S.lo[t][g] = (unsigned char)live;
                    S.hi[t][g] = (unsigned char)live;
                }
            }
            // queue the tests (order: entry, then i-cluster)
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const bool q = (need >> g) & 1u;
                const unsigned int b = __ballot_sync(0xffffffffu, q);
                const int base = S.ntest;
                if (q) S.test[base + __popc(b & ((1u << lane) - 1u))] = (unsigned short)(t | (g << 10));
                __syncwarp();
                if (lane == 0) S.ntest = base + __popc(b);
                __syncwarp();
            }
        }
        // (b) atom tests, lane per j row, four tests per pass
        const int n_t = S.ntest;
        const int jj = lane & 7, sub = lane >> 3;
        for (int u0 = 0; u0 < n_t; u0 += 4) {
            const int u = u0 + sub;
            bool in_lo = false, in_hi = false;
            int t = 0, g = 0;
            if (u < n_t) {
                const int code = S.test[u];
                t = code & 1023;
                g = code >> 10;
                const bool xm = t >= I.e_cnt;
                const unsigned int wd = S.word[t];
                const float4 s = S.sh[wd >> ROW_SLOT_BITS];
                const float4 xj = P.xq[(wd & ROW_SLOT_MASK) + jj];
                const float4 c = S.bb[g][0];
                const float jx = xj.x + s.x - c.x, jy = xj.y + s.y - c.y, jz = xj.z + s.z - c.z;
                // r^2 - r_in^2 = |x_j|^2 + (|x_i|^2 - r_in^2 - 2 x_i.x_j): the smallest of
                // the bracket over each half against -|x_j|^2
                const float njn = -fmaf(jx, jx, fmaf(jy, jy, jz * jz));
                unsigned int ex = 0u;
                if (xm) {
                    // excluded i atoms of this row: bits jj, jj + 8, ..., jj + 56 of the mask
                    const int k = I.x_begin + (t - I.e_cnt);
                    const unsigned long long m = P.xmasks[(size_t)k * GMAX + g];
#pragma unroll
                    for (int ii = 0; ii < CL; ++ii) ex |= (unsigned int)((m >> (ii * 8 + jj)) & 1ull) << ii;
                }
                float dm[2] = {3.0e38f, 3.0e38f};
#pragma unroll
                for (int ii = 0; ii < CL; ++ii) {
                    const float4 a = S.xi[g * CL + ii];
                    const float d = fmaf(a.x, jx, fmaf(a.y, jy, fmaf(a.z, jz, a.w)));
                    dm[ii >> 2] = fminf(dm[ii >> 2], ((ex >> ii) & 1u) ? 3.0e38f : d);
                }
                // a queued (entry, i-cluster) has both half tiles live: the outer
                // list is cluster-level
                in_lo = dm[0] < njn;
                in_hi = dm[1] < njn;
            }
            const unsigned int bl = __ballot_sync(0xffffffffu, in_lo);
            const unsigned int bh = __ballot_sync(0xffffffffu, in_hi);
            if (u < n_t && jj == 0) {
                S.lo[t][g] = (unsigned char)((bl >> (8 * sub)) & 0xFFu);
                S.hi[t][g] = (unsigned char)((bh >> (8 * sub)) & 0xFFu);
            }
        }
        __syncwarp();
        // pass 2: row counts per i-cluster: plain rows with both halves in
        // range (full), with only atoms 0-3 (lo) or only atoms 4-7 (hi), and
        // masked rows
        int cf[G], cl[G], ch[G], cx[G];
#pragma unroll
        for (int g = 0; g < G; ++g) { cf[g] = 0; cl[g] = 0; ch[g] = 0; cx[g] = 0; }
        for (int t = lane; t < n_e; t += 32) {
            const bool xm = t >= I.e_cnt;
            const int k = xm ? I.x_begin + (t - I.e_cnt) : I.e_begin + t;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const unsigned int lo = S.lo[t][g], hi = S.hi[t][g];
                unsigned int exr = 0u;
                if (xm) {
                    unsigned long long m = P.xmasks[(size_t)k * GMAX + g];
                    m |= m >> 32; m |= m >> 16; m |= m >> 8;
                    exr = (unsigned int)(m & 0xFFull);
                }
                cf[g] += __popc(lo & hi & ~exr);
                cl[g] += __popc(lo & ~hi & ~exr);
                ch[g] += __popc(hi & ~lo & ~exr);
                cx[g] += __popc((lo | hi) & exr);
            }
        }
        int totp = 0, totx = 0, nit = 0;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            for (int o = 16; o > 0; o >>= 1) {
                cf[g] += __shfl_xor_sync(0xffffffffu, cf[g], o);
                cl[g] += __shfl_xor_sync(0xffffffffu, cl[g], o);
                ch[g] += __shfl_xor_sync(0xffffffffu, ch[g], o);
                cx[g] += __shfl_xor_sync(0xffffffffu, cx[g], o);
            }
            totp += cf[g] + cl[g] + ch[g];
            totx += cx[g];
            nit += (cf[g] + cl[g] + ch[g] + cx[g]) > 0 ? 1 : 0;
        }
        if (nit == 0) continue;
        // offsets in this replica's regions
        unsigned int rb = 0u;
        int xb = 0, ib = 0;
        if (lane == 0) {
            rb = atomicAdd(&P.n_rows_r[I.rep], (unsigned int)totp);
            xb = atomicAdd(&P.n_xrows_r[I.rep], totx);
            ib = atomicAdd(&P.n_ritems_r[I.rep], nit);
        }
        rb = __shfl_sync(0xffffffffu, rb, 0);
        xb = __shfl_sync(0xffffffffu, xb, 0);
        ib = __shfl_sync(0xffffffffu, ib, 0);
        if ((long long)rb + totp > (long long)P.row_cap[I.rep] ||
            (long long)xb + totx > P.xrow_cap[I.rep] || (long long)ib + nit > P.ritem_cap[I.rep]) {
            if (lane == 0) {
                const int k = (long long)rb + totp > (long long)P.row_cap[I.rep] ? OVF_ROWS
                              : (long long)xb + totx > P.xrow_cap[I.rep]        ? OVF_XROWS
                                                                                : OVF_RITEMS;
                const long long need = k == OVF_ROWS ? (long long)rb + totp
                                       : k == OVF_XROWS ? (long long)xb + totx : (long long)ib + nit;
                set_err(P.cnt, ERRB_LIST, I.c0, (I.rep << 4) | k, (int)min(need, 2147483647LL));
            }
            continue;
        }
        rb += P.row_base[I.rep];
        xb += P.xrow_base[I.rep];
        ib += P.ritem_base[I.rep];
        // pass 3: write the rows (lane per entry, warp scans for the offsets) and
        // items. Per i-cluster: full rows, then rows with only atoms 0-3 in
        // range (lo), then rows with only atoms 4-7 (hi), each run in entry order.
        unsigned int ro = rb;
        int xo = xb, io = ib;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int nrow = cf[g] + cl[g] + ch[g];
            if (nrow + cx[g] == 0) continue;
            if (lane == 0) {
                RowItem ri;
                ri.c = I.c0 + g;
                ri.r_begin = ro;
                ri.x_begin = xo;
                ri.cnt = cf[g] | (cx[g] << 16);
                ri.n_lo = cl[g];
                ri.n_hi = ch[g];
                ri.pad0 = 0;
                ri.pad1 = 0;
                P.ritems[io] = ri;
            }
            ++io;
            const unsigned int lo_base = ro + (unsigned int)cf[g];
            const unsigned int hi_base = lo_base + (unsigned int)cl[g];
            int carf = 0, carl = 0, carh = 0, carx = 0;
            for (int t0 = 0; t0 < n_e; t0 += 32) {
                const int t = t0 + lane;
                unsigned int lo = 0u, hi = 0u, exr = 0u, base = 0u;
                unsigned long long m = 0ull;
                if (t < n_e) {
                    base = S.word[t];
                    lo = S.lo[t][g];
                    hi = S.hi[t][g];
                    if (t >= I.e_cnt) {
                        m = P.xmasks[(size_t)(I.x_begin + (t - I.e_cnt)) * GMAX + g];
                        unsigned long long f = m;
                        f |= f >> 32; f |= f >> 16; f |= f >> 8;
                        exr = (unsigned int)(f & 0xFFull);
                    }
                }
                const unsigned int mf = lo & hi & ~exr, ml = lo & ~hi & ~exr,
                                   mh = hi & ~lo & ~exr, mx = (lo | hi) & exr;
                const int nf = __popc(mf), nl = __popc(ml), nh = __popc(mh), nx = __popc(mx);
                int sf = nf, sl = nl, shh = nh, sx2 = nx;
                for (int o = 1; o < 32; o <<= 1) {
                    const int a0 = __shfl_up_sync(0xffffffffu, sf, o);
                    const int a1 = __shfl_up_sync(0xffffffffu, sl, o);
                    const int a2 = __shfl_up_sync(0xffffffffu, shh, o);
                    const int a3 = __shfl_up_sync(0xffffffffu, sx2, o);
                    if (lane >= o) { sf += a0; sl += a1; shh += a2; sx2 += a3; }
                }
                unsigned int of = ro + (unsigned int)(carf + sf - nf);
                unsigned int ol = lo_base + (unsigned int)(carl + sl - nl);
                unsigned int oh = hi_base + (unsigned int)(carh + shh - nh);
                int ox = xo + carx + sx2 - nx;
                for (int r = 0; r < CL; ++r) {
                    const unsigned int word = base + (unsigned int)r;
                    if ((mf >> r) & 1u) {
                        P.rows[of++] = word;
                    } else if ((ml >> r) & 1u) {
                        P.rows[ol++] = word;
                    } else if ((mh >> r) & 1u) {
                        P.rows[oh++] = word;
                    } else if ((mx >> r) & 1u) {
                        unsigned int em = 0u;
#pragma unroll
                        for (int ii = 0; ii < CL; ++ii)
                            em |= (unsigned int)((m >> (ii * 8 + r)) & 1ull) << ii;
                        P.xrows[ox++] = make_int2((int)word, (int)em);
                    }
                }
                carf += __shfl_sync(0xffffffffu, sf, 31);
                carl += __shfl_sync(0xffffffffu, sl, 31);
                carh += __shfl_sync(0xffffffffu, shh, 31);
                carx += __shfl_sync(0xffffffffu, sx2, 31);
            }
            ro += (unsigned int)nrow;
            xo += cx[g];
        }
    }
}

// Sums over replicas of two counts, to thread 0 of the block.
__device__ __forceinline__ void block_sum2(const void* a, bool a_unsigned, const int* b, int R,
                                           long long& ta, long long& tb) {
    __shared__ long long s_a[32], s_b[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = 0, y = 0;
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        x += a_unsigned ? (long long)((const unsigned int*)a)[r] : (long long)((const int*)a)[r];
        y += b[r];
    }
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    __syncthreads();
    if (lane == 0) { s_a[w] = x; s_b[w] = y; }
    __syncthreads();
    ta = tb = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { ta += s_a[k]; tb += s_b[k]; }
}

// After a prune: the prefix of the replicas' row-item counts (the pair
// kernels' iteration space) and the totals, in one block.
__global__ void __launch_bounds__(1024) k_prune_prefix(DevPtrs P) {
    if (!P.cnt->prune) return;
    const int n = block_prefix(P.n_ritems_r, P.ritem_cap, P.ritem_pref, P.R);
    __syncthreads();
    // the replica of the first item of every block of 256 items (the pair
    // kernels walk forward from it instead of searching the prefix)
    for (int b = threadIdx.x; b * 256 < n; b += blockDim.x) {
        const int it = b * 256;
        int lo = 0, hi = P.R - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.ritem_pref[mid] <= it) lo = mid;
            else hi = mid - 1;
        }
        P.ritem_blk[b] = lo;
    }
    long long rows = 0, xrows = 0;
    block_sum2(P.n_rows_r, true, P.n_xrows_r, P.R, rows, xrows);
    if (threadIdx.x == 0) {
        P.cnt->n_ritems = n;
        P.cnt->n_rows = (unsigned int)rows;
        P.cnt->n_xrows = (int)xrows;
    }
}

// After an outer build: the prefixes of the replicas' environment and ligand
// item counts and the totals.
__global__ void __launch_bounds__(1024) k_build_prefix(DevPtrs P) {
    if (!P.cnt->rebuild) return;
    const int ne = block_prefix(P.n_items_env_r, P.ienv_cap, P.ienv_pref, P.R);
    const int nl = block_prefix(P.n_items_lig_r, P.ilig_cap, P.ilig_pref, P.R);
    long long te = 0, tx = 0;
    block_sum2(P.n_entries_r, false, P.n_xentries_r, P.R, te, tx);
    if (threadIdx.x == 0) {
        P.cnt->n_items_env = ne;
        P.cnt->n_items_lig = nl;
        P.cnt->n_entries = (int)te;
        P.cnt->n_xentries = (int)tx;
    }
}

}  // namespace

void launch_rebuild(const DevPtrs& P, cudaStream_t s, int n_sm) {
    const int tb = 256;
    const int grid = max(1, min((P.S + tb - 1) / tb, n_sm * 8));
    k_rb_prepare<<<grid, tb, 0, s>>>(P);
    k_rb_colscan<<<P.R, 1024, 0, s>>>(P);
    k_rb_fill<<<grid, tb, 0, s>>>(P);
    k_rb_sort<<<(P.NCOL + SORT_WARPS - 1) / SORT_WARPS, SORT_WARPS * 32, 0, s>>>(P);
    k_rb_gather<<<grid, tb, 0, s>>>(P);
}

template <int G>
static void launch_lb_env(const DevPtrs& P, cudaStream_t s) {
    const size_t smem = sizeof(LBS<ENV_E, ENV_H, ENV_X, G>) * ENV_WARPS;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_build_list_env<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        attr = true;
    }
    static int grid = 0;
    if (!grid) {
        int dev = 0, n_sm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_list_env<G>, ENV_WARPS * 32,
                                                      smem);
        grid = n_sm * (per_sm > 0 ? per_sm : 1);
    }
    // about eight chunks per warp, at most 32 clusters each
    const int chunk = std::max(1, std::min(32, P.C / (grid * ENV_WARPS * 8)));
    k_build_list_env<G><<<grid, ENV_WARPS * 32, smem, s>>>(P, chunk);
}

void launch_list_build(const DevPtrs& P, cudaStream_t s, int max_lig_cl) {
    switch (P.group) {
        case 1: launch_lb_env<1>(P, s); break;
        case 2: launch_lb_env<2>(P, s); break;
        default: launch_lb_env<4>(P, s); break;
    }
    if (max_lig_cl > 0) {
        const size_t smem = sizeof(LBS<LIG_E, LIG_H, LIG_X, 1>) * LIG_WARPS;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_build_list_lig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            attr = true;
        }
        const int warps = P.R * max_lig_cl;
        k_build_list_lig<<<(warps + LIG_WARPS - 1) / LIG_WARPS, LIG_WARPS * 32, smem, s>>>(P, max_lig_cl);
    }
    k_build_prefix<<<1, 1024, 0, s>>>(P);
}

template <int G>
static void launch_prune_g(const DevPtrs& P, cudaStream_t s, int n_sm) {
    const size_t smem = sizeof(PrS<G>) * PR_WARPS;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_prune<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_prune<G><<<n_sm * 8, PR_WARPS * 32, smem, s>>>(P);
}

void launch_prune(const DevPtrs& P, cudaStream_t s, int n_sm) {
    const int tb = 256;
    const int grid = max(1, min((P.S + tb - 1) / tb, n_sm * 8));
    k_prune_prep<<<grid, tb, 0, s>>>(P);
    switch (P.group) {
        case 1: launch_prune_g<1>(P, s, n_sm); break;
        case 2: launch_prune_g<2>(P, s, n_sm); break;
        default: launch_prune_g<4>(P, s, n_sm); break;
    }
    k_prune_prefix<<<1, 1024, 0, s>>>(P);
}

}  // namespace abfe
