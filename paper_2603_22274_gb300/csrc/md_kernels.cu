// Integrator, bonded terms, restraint, reductions and output kernels.
//
// * k_integrate: one pass over all slots of all replicas: kick with the
//   fixed-point force, then (drift) A - O - A of BAOAB (Leimkuhler & Matthews
//   2013) with Philox4x32-10 normals (Salmon et al., SC'11) by Box-Muller,
//   clear the force accumulators, and the max squared displacement since the
//   last prune (drives the prune and rebuild decisions).
// * k_step_end: step counter, rebuild and prune flags, optional CUDA-graph
//   conditionals.
// * k_bonds: harmonic bonds (keep the synthetic molecules together).
// * k_boresch: the six-term Boresch restraint in FP64, one thread per replica
//   (paper, section "Restraints").
// * k_torsions: periodic torsions of the ligand's rotatable bonds, scaled by
//   lambda_v when annihilating (paper, section "Double annihilation protocol"),
//   FP64, one thread per torsion.
// * k_aw_refresh / k_aw_sums: alchemical waters (paper, section "Double
//   annihilation protocol"): their oxygens' slot charges at every replica's
//   lambda_q, and on energy passes the pair sums that give their part of
//   dU/dlambda_q and of u_kn.
// * k_finalize / k_ukn_assemble: fixed-point sums -> FP64 energies, dU/dlambda
//   and the reduced-potential row u_k = U(x; lambda_k) / kT.
#include <cuda_runtime.h>

#include "abfe_internal.cuh"

namespace abfe {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned int hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned int hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        if (r < 9) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
    }
    return c;
}

// three N(0,1) deviates for (atom, step, replica) under `seed`
__device__ __forceinline__ float3 gauss3(unsigned int atom, unsigned long long step,
                                         unsigned int replica, unsigned long long seed) {
    const uint4 x = philox4x32_10(
        make_uint4(atom, (unsigned int)step, (unsigned int)(step >> 32), replica),
        make_uint2((unsigned int)seed, (unsigned int)(seed >> 32)));
    const float k = 2.3283064365386963e-10f;  // 2^-32
    const float u0 = ((float)x.x + 0.5f) * k, u1 = ((float)x.y + 0.5f) * k;
    const float u2 = ((float)x.z + 0.5f) * k, u3 = ((float)x.w + 0.5f) * k;
    const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s0, c0, s1, c1;
    sincospif(2.0f * u1, &s0, &c0);
    sincospif(2.0f * u3, &s1, &c1);
    (void)s1;
    return make_float3(r0 * c0, r0 * s0, r1 * c1);
}

// Neighbour replica exchange (Hamiltonian exchange of lambda states): attempt
// t (Counters::ex_attempt) pairs the positions (m, m+1) of every group with
// m = t mod 2, 4, ... The
// pair's replicas ra (state a) and rb (state b) swap states with probability
// min(1, exp(-D)), D = [u_b(x_ra) + u_a(x_rb)] - [u_a(x_ra) + u_b(x_rb)], the
// Metropolis criterion of replica exchange in FP64 on the reduced potentials.
// The uniform: Philox4x32-10 at counter (t lo, t hi, group, m), key = seed,
// U = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53; accept iff D <= 0 or
// ln U < -D. Pairs are disjoint, so threads never touch the same replica.
__global__ void k_exchange(DevPtrs P, RepDev* reps, ExchangeDev X, const double* ukn, int ld,
                           unsigned long long seed) {
    const unsigned long long attempt = P.cnt->ex_attempt;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= X.R) return;
    const int g = X.grp[p];
    const int m = p - X.goff[g];
    if ((m & 1) != (int)(attempt & 1ull) || p + 1 >= X.goff[g + 1]) return;
    const int ra = X.slot_rep[p], rb = X.slot_rep[p + 1];
    const int a = X.held[p], b = X.held[p + 1];
    const double* ua = ukn + (size_t)ra * ld;
    const double* ub = ukn + (size_t)rb * ld;
    const double d = (ua[b] + ub[a]) - (ua[a] + ub[b]);
    const uint4 x = philox4x32_10(
        make_uint4((unsigned int)attempt, (unsigned int)(attempt >> 32), (unsigned int)g,
                   (unsigned int)m),
        make_uint2((unsigned int)seed, (unsigned int)(seed >> 32)));
    const double U = ((double)((unsigned long long)(x.x >> 5) * 67108864ull + (x.y >> 6)) + 0.5) *
                     1.1102230246251565e-16;  // 2^-53
    const bool acc = d <= 0.0 || log(U) < -d;
    if (!acc) return;
    X.slot_rep[p] = rb;
    X.slot_rep[p + 1] = ra;
    const int rr[2] = {ra, rb}, kk[2] = {b, a};
    for (int i = 0; i < 2; ++i) {
        RepDev& R = reps[rr[i]];
        const dbl4 st = P.sched_state[(size_t)R.sched * K_MAX + kk[i]];
        const double2 sc = X.sc[(size_t)R.sched * K_MAX + kk[i]];
        R.state = kk[i];
        R.dlam_r = st.x;
        R.dlam_q = st.y;
        R.dlam_v = st.z;
        R.lam_r = (float)st.x;
        R.lam_q = (float)st.y;
        R.lam_v = (float)st.z;
        R.dsc_A = sc.x;
        R.dsc_dA = sc.y;
        R.sc_A = (float)sc.x;
        R.sc_dA = (float)sc.y;
    }
    atomicAdd(X.n_acc, 1);
}

__global__ void k_exchange_done(Counters* c, const int* n_acc) {
    c->ex_attempt += 1ull;
    c->ex_accepted += *n_acc;
}

__device__ __forceinline__ float fixed_to_float(long long v) {
    return (float)((double)v * INV_FSCALE);
}

__global__ void __launch_bounds__(256) k_integrate(DevPtrs P) {
    const StepParams sp = *P.sp;
    const unsigned long long step = P.cnt->step;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P.cnt->env_next = 0;
        P.cnt->lig_next = 0;
    }
    // this step's energy sums start from zero
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.R * EA_N; i += gridDim.x * blockDim.x)
        P.eacc[i] = 0;
    const int lane = threadIdx.x & 31;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    float dmax = 0.0f, bmax = 0.0f;
    bool bad = false;
    for (int base = warp_global * 32; base < P.S; base += nwarps * 32) {
        const int s = base + lane;
        const int o = s < P.S ? P.orig[s] : -1;
        float d2 = 0.0f;   // squared displacement from the replica's prune positions
        float b2 = 0.0f;   // and from its outer-build positions
        if (o >= 0) {
            float4 x = P.xq[s];
            float4 v = P.v[s];
            const float invm = v.w;
            const float fxs = fixed_to_float(P.fx[s]), fys = fixed_to_float(P.fy[s]),
                        fzs = fixed_to_float(P.fz[s]);
            const float kk = sp.kick * invm;
            v.x = fmaf(kk, fxs, v.x);
            v.y = fmaf(kk, fys, v.y);
            v.z = fmaf(kk, fzs, v.z);
            if (sp.drift) {
                x.x = fmaf(sp.half_dt, v.x, x.x);
                x.y = fmaf(sp.half_dt, v.y, x.y);
                x.z = fmaf(sp.half_dt, v.z, x.z);
                const int rep = P.rep_of_cl[s >> 3];
                const float3 z = gauss3((unsigned int)o, step, (unsigned int)rep, sp.seed);
                const float sd = sp.c2 * sqrtf(invm);
                v.x = fmaf(sp.c1, v.x, sd * z.x);
                v.y = fmaf(sp.c1, v.y, sd * z.y);
                v.z = fmaf(sp.c1, v.z, sd * z.z);
                x.x = fmaf(sp.half_dt, v.x, x.x);
                x.y = fmaf(sp.half_dt, v.y, x.y);
                x.z = fmaf(sp.half_dt, v.z, x.z);
            }
            if (sp.zero_force) {
                P.fx[s] = 0; P.fy[s] = 0; P.fz[s] = 0;
            }
            if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) &&
                  isfinite(v.y) && isfinite(v.z)))
                bad = true;
            P.xq[s] = x;
            P.v[s] = v;
            const float4 r = P.xref[s], b = P.xbuild[s];
            const float dx = x.x - r.x, dy = x.y - r.y, dz = x.z - r.z;
            d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float bx = x.x - b.x, by = x.y - b.y, bz = x.z - b.z;
            b2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
        }
        dmax = fmaxf(dmax, d2);
        bmax = fmaxf(bmax, b2);
        // per replica: the largest over each cluster (8 lanes, one replica),
        // added once per warp when its 32 slots share a replica
        const int rep = s < P.S ? P.rep_of_cl[s >> 3] : -1;
        const bool one = __all_sync(FULL, rep == __shfl_sync(FULL, rep, 0));
        float m = d2, mb = b2;
        for (int k = 1; k < (one ? 32 : 8); k <<= 1) {
            m = fmaxf(m, __shfl_xor_sync(FULL, m, k));
            mb = fmaxf(mb, __shfl_xor_sync(FULL, mb, k));
        }
        if (rep >= 0 && (lane & (one ? 31 : 7)) == 0) {
            if (m > 0.0f) atomicMax(&P.disp_r[rep], __float_as_uint(m));
            if (mb > 0.0f) atomicMax(&P.dispb_r[rep], __float_as_uint(mb));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmaxf(dmax, __shfl_xor_sync(FULL, dmax, o));
        bmax = fmaxf(bmax, __shfl_xor_sync(FULL, bmax, o));
    }
    if (lane == 0 && dmax > 0.0f) atomicMax(&P.cnt->maxdisp2, __float_as_uint(dmax));
    if (lane == 0 && bmax > 0.0f) atomicMax(&P.cnt->dispb2, __float_as_uint(bmax));
    if (bad) set_err(P.cnt, ERRB_NONFINITE, -1);
}

// Step counter and the list decisions for this step, from the displacements
// the integrator measured: re-prune the inner list of every replica one of
// whose atoms now lies more than prune_skin/2 from its position at that
// replica's last prune; rebuild the outer list when an atom now lies more
// than skin/2 from its position at the outer build (the list holds every pair
// within r_c + skin there, so every pair within r_c now); a rebuild is always
// followed by a prune; both per replica (the replicas whose own atoms moved).
__global__ void __launch_bounds__(256) k_step_end(DevPtrs P, int inc_step, int force_rebuild,
                                                  int force_prune, cudaGraphConditionalHandle h_rb,
                                                  cudaGraphConditionalHandle h_pr,
                                                  cudaGraphConditionalHandle h_ex, int use_handle) {
    Counters* c = P.cnt;
    __shared__ int s_rb, s_pr;
    if (threadIdx.x == 0) {
        if (inc_step) c->step += 1ull;
        const float d2 = __uint_as_float(c->maxdisp2);
        const float db2 = __uint_as_float(c->dispb2);
        const bool nan = !(d2 == d2) || !(db2 == db2);
        const int rb = (force_rebuild || nan || db2 > P.skin_out_half2) ? 1 : 0;
        c->last_dispb2 = c->dispb2;
        c->dispb2 = 0u;     // both measured afresh by every step's integrator
        c->maxdisp2 = 0u;
        const int pr = (rb || force_prune || d2 > P.skin_in_half2) ? 1 : 0;
        c->rebuild = rb;
        c->prune = pr;
        if (pr) {
            c->prune_next = 0;
            c->n_prunes += 1;
        }
        s_rb = rb;
        s_pr = pr;
        if (use_handle) {
            cudaGraphSetConditional(h_rb, (unsigned int)rb);
            cudaGraphSetConditional(h_pr, (unsigned int)pr);
            // a replica-exchange attempt ends every ex_every-th step
            if (P.ex_every > 0)
                cudaGraphSetConditional(h_ex, (c->step % (unsigned long long)P.ex_every) == 0ull ? 1u : 0u);
        }
    }
    __syncthreads();
    // per replica: rebuilt in this step when any of its atoms left its half of
    // the outer skin (all replicas with a forced rebuild); pruned when it is
    // rebuilt, when any atom left its half of the prune skin, or with a forced
    // prune; the regions of the replicas rebuilt or pruned start empty
    int nb = 0, np = 0;
    // A window past 3/4 of either distance joins an update that another window
    // triggered (early updates are always exact): the updates of the windows
    // group into fewer events, each with fixed costs.
    constexpr float JOIN2 = 0.5625f;   // (3/4)^2
    for (int r = threadIdx.x; r < P.R; r += blockDim.x) {
        const float dr = __uint_as_float(P.disp_r[r]), db = __uint_as_float(P.dispb_r[r]);
        const int b = s_rb && (force_rebuild || !(db <= JOIN2 * P.skin_out_half2)) ? 1 : 0;
        const int f = s_pr && (b || force_prune || !(dr <= JOIN2 * P.skin_in_half2)) ? 1 : 0;
        P.bflag[r] = b;
        P.pflag[r] = f;
        P.disp_r[r] = 0u;
        P.dispb_r[r] = 0u;
        if (b) {
            P.n_entries_r[r] = 0;
            P.n_xentries_r[r] = 0;
            P.n_items_env_r[r] = 0;
            P.n_items_lig_r[r] = 0;
        }
        if (f) {
            P.n_rows_r[r] = 0u;
            P.n_xrows_r[r] = 0;
            P.n_ritems_r[r] = 0;
        }
        nb += b;
        np += f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        nb += __shfl_xor_sync(FULL, nb, o);
        np += __shfl_xor_sync(FULL, np, o);
    }
    if ((threadIdx.x & 31) == 0 && (nb || np)) {
        atomicAdd(&c->n_win_rebuilds, (unsigned long long)nb);
        atomicAdd(&c->n_win_prunes, (unsigned long long)np);
    }
}

template <typename T>
__device__ __forceinline__ T t_rint(T x);
template <>
__device__ __forceinline__ float t_rint<float>(float x) { return rintf(x); }
template <>
__device__ __forceinline__ double t_rint<double>(double x) { return rint(x); }

// Separation x_j - x_i at the nearest image, with the box length subtracted
// from the coordinate near it (exact), not from the difference: a bond across
// the wrap of the stored positions carries no rounding of a box-sized
// difference (which the stiff bonds would turn into ~0.1 kJ/mol/nm of force).
template <typename T>
__device__ __forceinline__ void bond_sep(const float4& xi, const float4& xj, const RepDev& R,
                                         T d[3]) {
    const float xiv[3] = {xi.x, xi.y, xi.z}, xjv[3] = {xj.x, xj.y, xj.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T L = (T)R.box[k], a = (T)xjv[k], b = (T)xiv[k];
        const T d0 = a - b;
        d[k] = d0 > (T)0.5 * L ? (a - L) - b : (d0 < (T)-0.5 * L ? a - (b - L) : d0);
    }
}

// harmonic bond: force on j along d is f d (on i: -f d), energy e
template <typename T>
__device__ __forceinline__ void bond_term(const T d[3], float2 pk, T& f, T& e) {
    const T r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const T dr = r - (T)pk.x;
    f = -(T)pk.y * dr / r;
    e = (T)0.5 * (T)pk.y * dr * dr;
}

// the bond's force on j in fixed point (on i: its negation, so a bond's pair
// of forces cancels exactly)
template <typename T>
__device__ __forceinline__ void bond_fixed(T f, const T d[3], long long v[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
        v[k] = sizeof(T) == 8 ? to_fixed_d((double)(f * d[k])) : to_fixed((float)(f * d[k]));
}

__device__ __forceinline__ void bond_add(const DevPtrs& P, int s, const long long v[3]) {
    add_fixed(P.fx + s, v[0]);
    add_fixed(P.fy + s, v[1]);
    add_fixed(P.fz + s, v[2]);
}

// One thread per bond unit of the flattened list over all replicas
// (bond_pref): a bonded triangle (the first n_bond_tri units of a replica,
// three bonds each) or a single bond. A block starts in replica
// bond_blk_rep[block] and its threads walk forward to their own replica, so no
// block idles on a small replica's bonds. Energies on energy steps only.
template <typename T, bool ENERGY>
__global__ void __launch_bounds__(256) k_bonds(DevPtrs P) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    int rep = P.bond_blk_rep[blockIdx.x];
    double e = 0.0;
    if (g < P.n_bond_total) {
        while (g >= P.bond_pref[rep + 1]) ++rep;
        const RepDev& R = P.reps[rep];
        const int u = g - P.bond_pref[rep];
        if (u < R.n_bond_tri) {
            const int b0 = R.bond_off + 3 * u;
            const int2 ab = P.sys_bond[b0], bc = P.sys_bond[b0 + 2];
            const float2 p_ab = P.sys_bond_p[b0], p_ac = P.sys_bond_p[b0 + 1],
                         p_bc = P.sys_bond_p[b0 + 2];
            const int sa = P.slot_of[R.atom_off + ab.x], sb = P.slot_of[R.atom_off + ab.y],
                      sc = P.slot_of[R.atom_off + bc.y];
            const float4 xa = P.xq[sa], xb = P.xq[sb], xc = P.xq[sc];
            T d_ab[3], d_ac[3], d_bc[3], f_ab, f_ac, f_bc, e_ab, e_ac, e_bc;
            bond_sep<T>(xa, xb, R, d_ab);
            bond_sep<T>(xa, xc, R, d_ac);
            bond_sep<T>(xb, xc, R, d_bc);
            bond_term<T>(d_ab, p_ab, f_ab, e_ab);
            bond_term<T>(d_ac, p_ac, f_ac, e_ac);
            bond_term<T>(d_bc, p_bc, f_bc, e_bc);
            // each bond's force rounded to fixed point on its own (as a lone
            // bond would be), then summed per atom in integers
            long long v_ab[3], v_ac[3], v_bc[3], Fa[3], Fb[3], Fc[3];
            bond_fixed<T>(f_ab, d_ab, v_ab);
            bond_fixed<T>(f_ac, d_ac, v_ac);
            bond_fixed<T>(f_bc, d_bc, v_bc);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Fa[k] = -v_ab[k] - v_ac[k];
                Fb[k] = v_ab[k] - v_bc[k];
                Fc[k] = v_ac[k] + v_bc[k];
            }
            bond_add(P, sa, Fa);
            bond_add(P, sb, Fb);
            bond_add(P, sc, Fc);
            if (ENERGY) e = (double)e_ab + (double)e_ac + (double)e_bc;
        } else {
            const int b = R.bond_off + 3 * R.n_bond_tri + (u - R.n_bond_tri);
            const int2 ij = P.sys_bond[b];
            const float2 pk = P.sys_bond_p[b];
            const int si = P.slot_of[R.atom_off + ij.x], sj = P.slot_of[R.atom_off + ij.y];
            T d[3], f, eb;
            bond_sep<T>(P.xq[si], P.xq[sj], R, d);
            bond_term<T>(d, pk, f, eb);
            long long Fj[3], Fi[3];
            bond_fixed<T>(f, d, Fj);
#pragma unroll
            for (int k = 0; k < 3; ++k) Fi[k] = -Fj[k];
            bond_add(P, sj, Fj);
            bond_add(P, si, Fi);
            if (ENERGY) e = (double)eb;
        }
    }
    if (!ENERGY) return;
    // bond energy per replica: a warp sum where the warp's bonds share one
    // replica, per-thread adds at replica boundaries (fixed point: the order
    // does not matter)
    const int rep0 = __shfl_sync(FULL, rep, 0);
    if (__all_sync(FULL, rep == rep0)) {
        double de = e;
        for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(FULL, de, o);
        if ((threadIdx.x & 31) == 0 && de != 0.0)
            add_fixed(P.eacc + (size_t)rep0 * EA_N + EA_BOND, to_fixed_d(de));
    } else if (e != 0.0) {
        add_fixed(P.eacc + (size_t)rep * EA_N + EA_BOND, to_fixed_d(e));
    }
}

// ------------------------------------------------------------------ Boresch (FP64)
struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3sub(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double d3dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 d3cross(D3 a, D3 b) {
    return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 d3scale(D3 a, double s) { return D3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ D3 d3add(D3 a, D3 b) { return D3{a.x + b.x, a.y + b.y, a.z + b.z}; }

// separation from atom `from` to atom `to`, nearest image
__device__ __forceinline__ D3 mi(const D3* p, int from, int to, const double* L) {
    D3 d = d3sub(p[to], p[from]);
    d.x -= L[0] * rint(d.x / L[0]);
    d.y -= L[1] * rint(d.y / L[1]);
    d.z -= L[2] * rint(d.z / L[2]);
    return d;
}

__global__ void k_boresch(DevPtrs P) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.R) return;
    const RepDev& R = P.reps[r];
    if (R.boresch < 0) {
        P.eb[r] = 0.0;
        return;
    }
    const BoreschDev B = P.bor[R.boresch];
    const double L[3] = {(double)R.box[0], (double)R.box[1], (double)R.box[2]};
    D3 p[6];
    int slot[6];
    for (int a = 0; a < 6; ++a) {
        slot[a] = P.slot_of[R.atom_off + B.anc[a]];
        const float4 x = P.xq[slot[a]];
        p[a] = D3{(double)x.x, (double)x.y, (double)x.z};
    }
    // anchor slots: 0 P1, 1 P2, 2 P3, 3 L1, 4 L2, 5 L3
    D3 grad[6];
    for (int a = 0; a < 6; ++a) grad[a] = D3{0, 0, 0};
    double U = 0.0;
    {   // distance P1-L1
        const D3 d = mi(p, 0, 3, L);
        const double rr = sqrt(d3dot(d, d));
        U += 0.5 * B.kr * (rr - B.r0) * (rr - B.r0);
        const D3 g = d3scale(d, B.kr * (rr - B.r0) / rr);
        grad[3] = d3add(grad[3], g);
        grad[0] = d3sub(grad[0], g);
    }
    // angles (outer a, vertex b, outer c): P1-L1-L2 and L1-P1-P2
    const int ang[2][3] = {{0, 3, 4}, {3, 0, 1}};
    for (int t = 0; t < 2; ++t) {
        const D3 u = mi(p, ang[t][1], ang[t][0], L), v = mi(p, ang[t][1], ang[t][2], L);
        const double lu = sqrt(d3dot(u, u)), lv = sqrt(d3dot(v, v));
        double c = d3dot(u, v) / (lu * lv);
        c = fmin(1.0, fmax(-1.0, c));
        const double th = acos(c);
        const double sn = sqrt(fmax(1.0 - c * c, 1e-300));
        const double dU = B.kth * (th - B.th0[t]);
        U += 0.5 * B.kth * (th - B.th0[t]) * (th - B.th0[t]);
        // d theta / d u = -(v/|v| - cos u/|u|) / (|u| sin)
        const D3 ga = d3scale(d3sub(d3scale(v, 1.0 / lv), d3scale(u, c / lu)), -1.0 / (lu * sn));
        const D3 gc = d3scale(d3sub(d3scale(u, 1.0 / lu), d3scale(v, c / lv)), -1.0 / (lv * sn));
        grad[ang[t][0]] = d3add(grad[ang[t][0]], d3scale(ga, dU));
        grad[ang[t][2]] = d3add(grad[ang[t][2]], d3scale(gc, dU));
        grad[ang[t][1]] = d3sub(grad[ang[t][1]], d3scale(d3add(ga, gc), dU));
    }
    // dihedrals a-b-c-d: P2-P1-L1-L2, P1-L1-L2-L3, L1-P1-P2-P3
    const int dih[3][4] = {{1, 0, 3, 4}, {0, 3, 4, 5}, {3, 0, 1, 2}};
    for (int t = 0; t < 3; ++t) {
        const D3 b1 = mi(p, dih[t][0], dih[t][1], L);
        const D3 b2 = mi(p, dih[t][1], dih[t][2], L);
        const D3 b3 = mi(p, dih[t][2], dih[t][3], L);
        const D3 n1 = d3cross(b1, b2), n2 = d3cross(b2, b3);
        const double lb2 = sqrt(d3dot(b2, b2));
        const double phi = atan2(lb2 * d3dot(b1, n2), d3dot(n1, n2));
        const double dU = B.kph * sin(phi - B.ph0[t]);
        U += B.kph * (1.0 - cos(phi - B.ph0[t]));
        const D3 ga = d3scale(n1, -lb2 / d3dot(n1, n1));
        const D3 gd = d3scale(n2, lb2 / d3dot(n2, n2));
        const double pp = d3dot(b1, b2) / (lb2 * lb2), qq = d3dot(b3, b2) / (lb2 * lb2);
        const D3 gb = d3add(d3scale(ga, -(1.0 + pp)), d3scale(gd, qq));
        const D3 gc = d3add(d3scale(ga, pp), d3scale(gd, -(1.0 + qq)));
        grad[dih[t][0]] = d3add(grad[dih[t][0]], d3scale(ga, dU));
        grad[dih[t][1]] = d3add(grad[dih[t][1]], d3scale(gb, dU));
        grad[dih[t][2]] = d3add(grad[dih[t][2]], d3scale(gc, dU));
        grad[dih[t][3]] = d3add(grad[dih[t][3]], d3scale(gd, dU));
    }
    const double lr = R.dlam_r;
    if (lr != 0.0) {
        for (int a = 0; a < 6; ++a) {
            add_fixed(P.fx + slot[a], to_fixed_d(-lr * grad[a].x));
            add_fixed(P.fy + slot[a], to_fixed_d(-lr * grad[a].y));
            add_fixed(P.fz + slot[a], to_fixed_d(-lr * grad[a].z));
        }
    }
    if (!isfinite(U)) set_err(P.cnt, ERRB_NONFINITE, r);
    P.eb[r] = U;
}

// U = s sum_t k_t [1 + cos(n_t phi_t - phi0_t)], s = lambda_v (annihilation)
// or 1 (decoupling); phi from b1 = x_b - x_a, b2 = x_c - x_b, b3 = x_d - x_c
// (nearest images) as atan2(|b2| b1.(b2 x b3), (b1 x b2).(b2 x b3)). The
// gradient: d phi/d x_a = -|b2| n1/|n1|^2, d phi/d x_d = |b2| n2/|n2|^2 and the
// inner atoms from those with the projections b1.b2/|b2|^2 and b3.b2/|b2|^2.
// The unscaled sum goes to EA_TORS, and (annihilation) to dU/dlambda_v.
__global__ void __launch_bounds__(128) k_torsions(DevPtrs P) {
    const int rep = blockIdx.y;
    const RepDev& R = P.reps[rep];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (t < R.n_tors) {
        const int4 q = P.sys_tors[R.tors_off + t];
        const dbl4 prm = P.sys_torsp[R.tors_off + t];
        const int sl[4] = {P.slot_of[R.atom_off + q.x], P.slot_of[R.atom_off + q.y],
                           P.slot_of[R.atom_off + q.z], P.slot_of[R.atom_off + q.w]};
        D3 p[4];
        for (int a = 0; a < 4; ++a) {
            const float4 x = P.xq[sl[a]];
            p[a] = D3{(double)x.x, (double)x.y, (double)x.z};
        }
        const double L[3] = {(double)R.box[0], (double)R.box[1], (double)R.box[2]};
        const D3 b1 = mi(p, 0, 1, L), b2 = mi(p, 1, 2, L), b3 = mi(p, 2, 3, L);
        const D3 n1 = d3cross(b1, b2), n2 = d3cross(b2, b3);
        const double lb2 = sqrt(d3dot(b2, b2));
        const double phi = atan2(lb2 * d3dot(b1, n2), d3dot(n1, n2));
        const double arg = prm.y * phi - prm.z;
        e = prm.x * (1.0 + cos(arg));
        const bool ann = P.ligand_mode == 0;
        const double s = ann ? R.dlam_v : 1.0;
        // dU/dphi of the state
        const double dU = -s * prm.x * prm.y * sin(arg);
        if (dU != 0.0) {
            const D3 ga = d3scale(n1, -lb2 / d3dot(n1, n1));
            const D3 gd = d3scale(n2, lb2 / d3dot(n2, n2));
            const double pp = d3dot(b1, b2) / (lb2 * lb2), qq = d3dot(b3, b2) / (lb2 * lb2);
            const D3 g[4] = {ga, d3add(d3scale(ga, -(1.0 + pp)), d3scale(gd, qq)),
                             d3add(d3scale(ga, pp), d3scale(gd, -(1.0 + qq))), gd};
            for (int a = 0; a < 4; ++a) {
                add_fixed(P.fx + sl[a], to_fixed_d(-dU * g[a].x));
                add_fixed(P.fy + sl[a], to_fixed_d(-dU * g[a].y));
                add_fixed(P.fz + sl[a], to_fixed_d(-dU * g[a].z));
            }
        }
    }
    __shared__ double s_e[4];
    double de = e;
    for (int o = 16; o > 0; o >>= 1) de += __shfl_xor_sync(FULL, de, o);
    if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = de;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += s_e[w];
        if (!isfinite(tt)) set_err(P.cnt, ERRB_NONFINITE, rep);
        if (tt != 0.0) {
            add_fixed(P.eacc + (size_t)rep * EA_N + EA_TORS, to_fixed_d(tt));
            if (P.ligand_mode == 0) add_fixed(P.eacc + (size_t)rep * EA_N + EA_DUDLV, to_fixed_d(tt));
        }
    }
}

// Slot charges of the alchemical oxygens at each replica's lambda_q (the same
// float expression as the list rebuild's gather, so a state changed here and a
// state set before a rebuild give identical charges). One block per replica.
__global__ void k_aw_refresh(DevPtrs P) {
    const RepDev& R = P.reps[blockIdx.x];
    for (int k = threadIdx.x; k < R.n_aw; k += blockDim.x) {
        const int o = P.sys_aw[R.aw_off + k];
        const int s = P.slot_of[R.atom_off + o];
        float4 x = P.xq[s];
        x.w = fmaf(1.0f - R.lam_q, P.sys_dq[R.sys_atom_off + o], P.sys_prm[R.sys_atom_off + o].x);
        P.xq[s] = x;
    }
}

// Energy passes: for alchemical oxygen a (block (a, replica)) the pairs with
// every atom j of its window within the cutoff, not excluded, in FP64 with
// f = k_e erfc(beta r) / r and the base charges q0 (e): A2 += dq_a q0_j f for j
// neither ligand nor alchemical, B2 += dq_a q0_j f for ligand j, and for an
// alchemical j = b > a: C01 += (q0_a dq_b + dq_a q0_b) f, C11 += dq_a dq_b f.
__global__ void __launch_bounds__(128) k_aw_sums(DevPtrs P) {
    const int rep = blockIdx.y;
    const RepDev& R = P.reps[rep];
    const int k = blockIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (k < R.n_aw) {
        const int a = P.sys_aw[R.aw_off + k];
        const int sa = P.slot_of[R.atom_off + a];
        const float4 xa = P.xq[sa];
        const double q0a = P.sys_prmd[R.sys_atom_off + a].x, dqa = P.sys_dqd[R.sys_atom_off + a];
        const int eb = P.sys_ex_off[R.sys_ex_off + a], ee = P.sys_ex_off[R.sys_ex_off + a + 1];
        const double L[3] = {(double)R.box[0], (double)R.box[1], (double)R.box[2]};
        const int s0 = R.cl_off * CL, s1 = (R.cl_off + R.n_cl_cap) * CL;
        for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
            const int o = P.orig[s];
            if (o < 0 || o == a) continue;
            bool ex = false;
            for (int q = eb; q < ee; ++q) ex |= P.sys_ex_idx[q] == o;
            if (ex) continue;
            const float4 xj = P.xq[s];
            double d[3] = {(double)xj.x - xa.x, (double)xj.y - xa.y, (double)xj.z - xa.z};
            for (int c = 0; c < 3; ++c) d[c] -= L[c] * rint(d[c] / L[c]);
            const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < P.drc2)) continue;
            const double r = sqrt(r2);
            const double f = P.dke * erfc(P.dbeta * r) / r;
            const double q0j = P.sys_prmd[R.sys_atom_off + o].x;
            const double dqj = P.sys_dqd[R.sys_atom_off + o];
            if (P.sys_lig[R.sys_atom_off + o]) {
                acc[1] += dqa * q0j * f;
            } else if (dqj != 0.0) {
                if (o > a) {
                    acc[2] += (q0a * dqj + dqa * q0j) * f;
                    acc[3] += dqa * dqj * f;
                }
            } else {
                acc[0] += dqa * q0j * f;
            }
        }
    }
    __shared__ double s_acc[4][4];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) s_acc[wp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4 && k < R.n_aw) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_acc[w][threadIdx.x];
        if (!isfinite(v)) set_err(P.cnt, ERRB_NONFINITE, rep);
        if (v != 0.0) add_fixed(P.eacc + (size_t)rep * EA_N + EA_AW_A2 + threadIdx.x, to_fixed_d(v));
    }
}

__global__ void k_finalize(DevPtrs P) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.R) return;
    const RepDev& R = P.reps[r];
    const long long* a = P.eacc + (size_t)r * EA_N;
    double E[ABFE_N_ENERGY];
    E[ABFE_E_ENV_LJ] = (double)a[EA_ENV_LJ] * INV_FSCALE;
    E[ABFE_E_ENV_COUL] = (double)a[EA_ENV_C] * INV_FSCALE;
    E[ABFE_E_LIGENV_LJ] = (double)a[EA_LIGENV_LJ] * INV_FSCALE;
    E[ABFE_E_LIGLIG_LJ] = (double)a[EA_LIGLIG_LJ] * INV_FSCALE;
    E[ABFE_E_LIGENV_COUL] = (double)a[EA_LIGENV_C] * INV_FSCALE;
    E[ABFE_E_LIGLIG_COUL] = (double)a[EA_LIGLIG_C] * INV_FSCALE;
    E[ABFE_E_BOND] = (double)a[EA_BOND] * INV_FSCALE;
    E[ABFE_E_RESTRAINT] = R.dlam_r * P.eb[r];
    E[ABFE_E_RECIP] = 0.0;
    E[ABFE_E_TORSION] = (P.ligand_mode == 0 ? R.dlam_v : 1.0) * ((double)a[EA_TORS] * INV_FSCALE);
    double dq_pme = 0.0;
    if (P.pme) {
        // reciprocal + excluded-pair energies at lambda_q, self energy; dU/dlambda_q
        // from the decomposition E_rec = A + lambda B + lambda^2 C (energy passes)
        const double2 sf = P.pme_self[R.sys];
        const double lq = R.dlam_q;
        E[ABFE_E_RECIP] = ((double)a[EA_REC] + (double)a[EA_EXCL]) * INV_FSCALE + sf.x + lq * lq * sf.y;
        const double A = (double)a[EA_REC_ENV] * INV_FSCALE, C = (double)a[EA_REC_LIG] * INV_FSCALE;
        const double B = (double)a[EA_REC_MIX] * INV_FSCALE;
        dq_pme = B + 2.0 * lq * (C + sf.y + (double)a[EA_EXCL_LIG] * INV_FSCALE) +
                 (double)a[EA_EXCL_MIX] * INV_FSCALE;
    }
    double t = 0.0;
    for (int k = 0; k < ABFE_E_TOTAL; ++k) t += E[k];
    E[ABFE_E_TOTAL] = t;
    if (P.out_energy)
        for (int k = 0; k < ABFE_N_ENERGY; ++k) P.out_energy[(size_t)r * ABFE_N_ENERGY + k] = E[k];
    if (P.out_dudl) {
        P.out_dudl[(size_t)r * ABFE_N_DUDL + ABFE_DUDL_RESTRAINT] = P.eb[r];
        // alchemical waters: the pair kernels saw their charges at this state; the
        // derivative of E_aw(lambda) = (1-l) A2 + l (1-l) B2 + (1-l) C01 + (1-l)^2 C11
        // + lambda-independent terms, less the part the ligand pairs already hold
        double dq_aw = 0.0;
        if (R.n_aw > 0) {
            const double l0 = R.dlam_q;
            dq_aw = -l0 * (double)a[EA_AW_B2] * INV_FSCALE - (double)a[EA_AW_A2] * INV_FSCALE -
                    (double)a[EA_AW_C01] * INV_FSCALE -
                    2.0 * (1.0 - l0) * (double)a[EA_AW_C11] * INV_FSCALE;
        }
        P.out_dudl[(size_t)r * ABFE_N_DUDL + ABFE_DUDL_COUL] =
            (double)a[EA_DUDLQ] * INV_FSCALE + dq_pme + dq_aw;
        P.out_dudl[(size_t)r * ABFE_N_DUDL + ABFE_DUDL_VDW] = (double)a[EA_DUDLV] * INV_FSCALE;
    }
}

__global__ void k_ukn_assemble(DevPtrs P, double kT) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P.R * P.ukn_ld) return;
    const int r = idx / P.ukn_ld, k = idx % P.ukn_ld;
    const RepDev& R = P.reps[r];
    const int K = P.sched_K[R.sched];
    if (k >= K) {
        P.out_ukn[idx] = 0.0;
        if (P.out_du) P.out_du[idx] = 0.0;
        return;
    }
    const long long* a = P.eacc + (size_t)r * EA_N;
    const bool dec = P.ligand_mode == 1;
    double e_indep = ((double)a[EA_ENV_LJ] + (double)a[EA_ENV_C] + (double)a[EA_BOND]) * INV_FSCALE;
    const double ut = (double)a[EA_TORS] * INV_FSCALE;   // rotatable-bond torsions, unscaled
    if (dec) e_indep += ((double)a[EA_LIGLIG_LJ] + (double)a[EA_LIGLIG_C]) * INV_FSCALE + ut;
    const dbl4 st = P.sched_state[R.sched * K_MAX + k];
    const int kv = (int)st.w;
    const double cle = (double)P.ukn_c[(size_t)r * 2 + 0] * INV_FSCALE;
    const double cll = (double)P.ukn_c[(size_t)r * 2 + 1] * INV_FSCALE;
    const double lj = (double)P.ukn_lj[(size_t)r * KV_MAX + kv] * INV_FSCALE;
    double du = st.x * P.eb[r] + st.y * cle + (dec ? 0.0 : st.y * st.y * cll + st.z * ut) + lj;
    if (R.n_aw > 0) {
        // alchemical waters: the pair sums at this replica's lambda_q (l0) hold
        // their pairs at l0; move them to state k's lambda_q (lk)
        const double l0 = R.dlam_q, lk = st.y;
        const double A2 = (double)a[EA_AW_A2] * INV_FSCALE, B2 = (double)a[EA_AW_B2] * INV_FSCALE;
        const double C01 = (double)a[EA_AW_C01] * INV_FSCALE, C11 = (double)a[EA_AW_C11] * INV_FSCALE;
        e_indep -= (1.0 - l0) * (A2 + C01) + (1.0 - l0) * (1.0 - l0) * C11;
        du += lk * (l0 - lk) * B2 + (1.0 - lk) * (A2 + C01) + (1.0 - lk) * (1.0 - lk) * C11;
    }
    if (P.pme) {
        // reciprocal part: A + lambda_q B + lambda_q^2 C, self and excluded pairs by kind
        const double2 sf = P.pme_self[R.sys];
        const double A = (double)a[EA_REC_ENV] * INV_FSCALE, C = (double)a[EA_REC_LIG] * INV_FSCALE;
        const double B = (double)a[EA_REC_MIX] * INV_FSCALE;
        const double lq = st.y;
        e_indep += A + sf.x + (double)a[EA_EXCL_ENV] * INV_FSCALE;
        du += lq * (B + (double)a[EA_EXCL_MIX] * INV_FSCALE) +
              lq * lq * (C + sf.y + (double)a[EA_EXCL_LIG] * INV_FSCALE);
    }
    P.out_ukn[idx] = (e_indep + du) / kT;
    if (P.out_du) P.out_du[idx] = du;
}

// per slot: scatter a per-atom quantity to original order
// what: 0 forces (double), 1 forces (float), 2 positions, 3 velocities,
// 4 positions at the last prune, 5 positions at the last outer list build
__global__ void k_scatter_out(DevPtrs P, int what, double* outd, float* outf) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        const int o = P.orig[s];
        if (o < 0) continue;
        const RepDev& R = P.reps[P.rep_of_cl[s >> 3]];
        const size_t row = (size_t)(R.atom_off + o) * 3;
        double v0, v1, v2;
        if (what <= 1) {
            v0 = (double)P.fx[s] * INV_FSCALE;
            v1 = (double)P.fy[s] * INV_FSCALE;
            v2 = (double)P.fz[s] * INV_FSCALE;
        } else if (what == 2) {
            const float4 x = P.xq[s];
            v0 = x.x; v1 = x.y; v2 = x.z;
        } else if (what == 4) {
            const float4 x = P.xref[s];
            v0 = x.x; v1 = x.y; v2 = x.z;
        } else if (what == 5) {
            const float4 x = P.xbuild[s];
            v0 = x.x; v1 = x.y; v2 = x.z;
        } else {
            const float4 v = P.v[s];
            v0 = v.x; v1 = v.y; v2 = v.z;
        }
        if (what == 1) {
            outf[row] = (float)v0; outf[row + 1] = (float)v1; outf[row + 2] = (float)v2;
        } else {
            outd[row] = v0; outd[row + 1] = v1; outd[row + 2] = v2;
        }
    }
}

// per slot: read positions (what 2) or velocities (what 3) from original order
__global__ void k_gather_in(DevPtrs P, int what, const double* in) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        const int o = P.orig[s];
        if (o < 0) continue;
        const RepDev& R = P.reps[P.rep_of_cl[s >> 3]];
        const size_t row = (size_t)(R.atom_off + o) * 3;
        if (what == 2) {
            float4 x = P.xq[s];
            x.x = (float)in[row]; x.y = (float)in[row + 1]; x.z = (float)in[row + 2];
            P.xq[s] = x;
        } else {
            float4 v = P.v[s];
            v.x = (float)in[row]; v.y = (float)in[row + 1]; v.z = (float)in[row + 2];
            P.v[s] = v;
        }
    }
}

}  // namespace

void launch_integrate(const DevPtrs& P, cudaStream_t s, int n_sm) {
    const int tb = 256;
    const int grid = max(1, min((P.S + tb - 1) / tb, n_sm * 8));
    k_integrate<<<grid, tb, 0, s>>>(P);
}

void launch_step_end(const DevPtrs& P, cudaStream_t s, int inc_step, int force_rebuild,
                     int force_prune, cudaGraphConditionalHandle h_rebuild,
                     cudaGraphConditionalHandle h_prune, cudaGraphConditionalHandle h_exchange,
                     int use_handle) {
    k_step_end<<<1, 256, 0, s>>>(P, inc_step, force_rebuild, force_prune, h_rebuild, h_prune,
                               h_exchange, use_handle);
}

void launch_bonds(const DevPtrs& P, cudaStream_t s, int precision, bool energy) {
    if (P.n_bond_total <= 0) return;
    const int grid = (P.n_bond_total + 255) / 256;
    if (precision == 1) {
        if (energy) k_bonds<double, true><<<grid, 256, 0, s>>>(P);
        else k_bonds<double, false><<<grid, 256, 0, s>>>(P);
    } else {
        if (energy) k_bonds<float, true><<<grid, 256, 0, s>>>(P);
        else k_bonds<float, false><<<grid, 256, 0, s>>>(P);
    }
}

void launch_torsions(const DevPtrs& P, cudaStream_t s, int max_tors) {
    if (max_tors <= 0) return;
    dim3 grid((max_tors + 127) / 128, P.R);
    k_torsions<<<grid, 128, 0, s>>>(P);
}

void launch_aw_refresh(const DevPtrs& P, cudaStream_t s) {
    k_aw_refresh<<<P.R, 32, 0, s>>>(P);
}

void launch_aw_sums(const DevPtrs& P, cudaStream_t s, int max_aw) {
    if (max_aw <= 0) return;
    k_aw_sums<<<dim3(max_aw, P.R), 128, 0, s>>>(P);
}

void launch_boresch(const DevPtrs& P, cudaStream_t s) {
    k_boresch<<<(P.R + 63) / 64, 64, 0, s>>>(P);
}

void launch_finalize(const DevPtrs& P, cudaStream_t s) {
    k_finalize<<<(P.R + 127) / 128, 128, 0, s>>>(P);
}

void launch_ukn_assemble(const DevPtrs& P, cudaStream_t s, double kT) {
    const int n = P.R * P.ukn_ld;
    k_ukn_assemble<<<(n + 255) / 256, 256, 0, s>>>(P, kT);
}

void launch_scatter_out(const DevPtrs& P, cudaStream_t s, int what, double* outd, float* outf,
                        int n_sm) {
    const int grid = max(1, min((P.S + 255) / 256, n_sm * 8));
    k_scatter_out<<<grid, 256, 0, s>>>(P, what, outd, outf);
}

void launch_gather_in(const DevPtrs& P, cudaStream_t s, int what, const double* in, int n_sm) {
    const int grid = max(1, min((P.S + 255) / 256, n_sm * 8));
    k_gather_in<<<grid, 256, 0, s>>>(P, what, in);
}

void launch_exchange(const DevPtrs& P, RepDev* reps, const ExchangeDev& X, const double* ukn, int ld,
                     unsigned long long seed, cudaStream_t s) {
    cudaMemsetAsync(X.n_acc, 0, sizeof(int), s);
    k_exchange<<<(X.R + 127) / 128, 128, 0, s>>>(P, reps, X, ukn, ld, seed);
    k_exchange_done<<<1, 1, 0, s>>>(P.cnt, X.n_acc);
    if (P.has_aw) k_aw_refresh<<<P.R, 32, 0, s>>>(P);   // new lambda_q: alchemical charges
}

}  // namespace abfe
