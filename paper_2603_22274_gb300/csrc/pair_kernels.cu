// Nonbonded pair kernels.
//
// * k_env_rows: environment-environment pairs (lambda independent): plain
//   12-6 LJ with Lorentz-Berthelot mixing plus real-space Ewald Coulomb, hard
//   cutoff, over the inner list of j rows. A warp owns one i-cluster (8 atoms,
//   held in shared memory) and walks its rows 32 at a time, a lane per row:
//   the lane loads the row's j atom once and evaluates it against the i atoms
//   the row covers (all 8 of a full row; atoms 0-3 or 4-7 of a half row, the
//   rows being ordered full | lower half | upper half so that most rounds
//   skip the unused half block for the whole warp); its j force goes to the
//   64-bit fixed-point accumulators once per row and the i forces stay in
//   registers until the item ends. FP32 forces: the Coulomb force is
//   qq G(r) / r^3 with G from a quadratic table in r held in shared memory
//   (ewald_G); FP32 energies (energy steps only) use correctly rounded
//   arithmetic and erfcf/expf; FP64 uses erfc/exp.
// * k_lig: ligand-involved pairs at the replica's own state (outer list, 4x8
//   half tiles: lane = jj + 8 ii): Beutler softcore LJ, lambda_q-scaled
//   charges, dU/dlambda_v and dU/dlambda_q; pair arithmetic in the kernel's
//   precision, energy sums (energy steps only) in FP64.
// * k_lig_ukn: the same pairs at every distinct lambda_v of the replica's
//   schedule, plus the unit-charge Coulomb sums, for the u_kn row.
// * k_count_rows / k_count: in-cutoff pair counts through the inner rows and the
//   ligand list (list parity checks) and the computed pair lanes.
#include <cuda_runtime.h>

#include "abfe_internal.cuh"

namespace abfe {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <typename T>
struct T3 {
    T x, y, z;
};

template <typename T>
struct Atom {
    T x, y, z, q, sh, e2;  // position, q sqrt(ke), sigma/2, 2 sqrt(eps)
};

template <typename T>
struct KC {
    T rc2, beta, tbsp, nb2l2e, dke_sqrt;
    const float4* tab;   // FP32 path: the Ewald force table in shared memory
    float inv_h;
};

template <typename T>
__device__ __forceinline__ KC<T> make_kc(const DevPtrs& P);
template <>
__device__ __forceinline__ KC<float> make_kc<float>(const DevPtrs& P) {
    return KC<float>{P.rc2, P.beta, P.tbsp, P.nb2l2e, P.sqrt_ke, nullptr, P.ewtab_inv_h};
}
template <>
__device__ __forceinline__ KC<double> make_kc<double>(const DevPtrs& P) {
    return KC<double>{P.drc2, P.dbeta, 2.0 * P.dbeta / sqrt(3.14159265358979323846), 0.0,
                      sqrt(P.dke), nullptr, 0.0f};
}

template <typename T>
__device__ __forceinline__ Atom<T> load_atom(const DevPtrs& P, int slot, const RepDev& R,
                                             const KC<T>& K);
template <>
__device__ __forceinline__ Atom<float> load_atom<float>(const DevPtrs& P, int slot, const RepDev&,
                                                        const KC<float>&) {
    const float4 x = P.xq[slot];
    const float2 s = P.se[slot];
    return Atom<float>{x.x, x.y, x.z, x.w, s.x, s.y};
}
template <>
__device__ __forceinline__ Atom<double> load_atom<double>(const DevPtrs& P, int slot,
                                                          const RepDev& R, const KC<double>& K) {
    const float4 x = P.xq[slot];
    const int o = P.orig[slot];
    Atom<double> a{(double)x.x, (double)x.y, (double)x.z, 0.0, 0.0, 0.0};
    if (o >= 0) {
        const int sys_atom_off = R.sys_atom_off;
        const dbl4 p = P.sys_prmd[sys_atom_off + o];
        // alchemical oxygens: q0 + (1 - lambda_q) dq
        a.q = fma(1.0 - R.dlam_q, P.sys_dqd[sys_atom_off + o], p.x) * K.dke_sqrt;
        a.sh = 0.5 * p.y;
        a.e2 = 2.0 * sqrt(p.z);
    }
    return a;
}

__device__ __forceinline__ float t_rsqrt(float x) { return rsqrt_fast(x); }
__device__ __forceinline__ double t_rsqrt(double x) { return rsqrt(x); }

// erfc(beta r) and exp(-beta^2 r^2)
__device__ __forceinline__ void ewald(double r, double r2, const KC<double>& K, double& erfcv,
                                      double& ex) {
    ex = exp(-K.beta * K.beta * r2);
    erfcv = erfc(K.beta * r);
}

// G(r) from the shared-memory table: the nearest grid point j = round(t),
// t = r / h (clamped to the table), and the centred quadratic in f = t - j.
// Adding 1.5 * 2^23 leaves round(t) in the low mantissa bits (t < 2^22), so no
// conversion instruction is needed.
__device__ __forceinline__ float ewald_G(float r, const float4* tab, float inv_h) {
    const float t = fminf(r * inv_h, (float)(EW_NT - 1));
    const float tr = t + 12582912.0f;
    const int j = __float_as_int(tr) - 0x4B400000;
    const float f = t - (tr - 12582912.0f);
    const float4 c = tab[j];
    return fmaf(fmaf(c.z, f, c.y), f, c.x);
}

// correctly rounded / library-accurate variants, used where energies are
// summed for dU/dlambda and u_kn (ligand pairs, energy steps)
__device__ __forceinline__ float t_sqrt_acc(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ double t_sqrt_acc(double x) { return sqrt(x); }
__device__ __forceinline__ float t_rcp_acc(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double t_rcp_acc(double x) { return 1.0 / x; }
__device__ __forceinline__ void ewald_acc(float r, float r2, const KC<float>& K, float& erfcv,
                                          float& ex) {
    ex = expf(-(K.beta * K.beta) * r2);
    erfcv = erfcf(K.beta * r);
}
__device__ __forceinline__ void ewald_acc(double r, double r2, const KC<double>& K, double& erfcv,
                                          double& ex) {
    ewald(r, r2, K, erfcv, ex);
}

// x_j + s - c (image shift s, reference atom c of the i-cluster): the box
// length is only subtracted from a coordinate near it (exact), so an image
// pair's separation carries no rounding of a box-sized sum
template <typename T>
__device__ __forceinline__ T rel_img(float xj, float s, float c) {
    return s > 0.f ? (T)xj + (T)(s - c) : ((T)xj + (T)s) - (T)c;
}

// Inner-list item `it` of the iteration space over all replicas' regions: from
// the replica of its block of 256 items, forward to the last replica r with
// ritem_pref[r] <= it (an empty replica shares its successor's prefix).
__device__ __forceinline__ const RowItem& row_item(const DevPtrs& P, int it) {
    int r = P.ritem_blk[it >> 8];
    while (r + 1 < P.R && P.ritem_pref[r + 1] <= it) ++r;
    return P.ritems[P.ritem_base[r] + (it - P.ritem_pref[r])];
}

// ------------------------------------------------------------------ env pair
template <typename T, bool ENERGY>
__device__ __forceinline__ void pair_env(const Atom<T>& ai, const Atom<T>& aj, bool keep,
                                         T3<T>& fi, T3<T>& fj, T& elj, T& ec, const KC<T>& K) {
    const T dx = aj.x - ai.x, dy = aj.y - ai.y, dz = aj.z - ai.z;
    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    keep = keep && (r2 < K.rc2);
    const T rinv = t_rsqrt(r2);
    const T rinv2 = rinv * rinv;
    const T qq = ai.q * aj.q;
    T fcr;  // Coulomb force times r^2
    if constexpr (sizeof(T) == 4) {
        // Coulomb force qq G(r) / r^3 from the table
        fcr = qq * ewald_G(r2 * rinv, K.tab, K.inv_h) * rinv;
    } else {
        const T r = r2 * rinv;
        T erfcv, ex;
        ewald(r, r2, K, erfcv, ex);
        const T vc = qq * erfcv * rinv;
        fcr = fma(qq * K.tbsp, ex, vc);
    }
    const T sig = ai.sh + aj.sh;
    const T eps4 = ai.e2 * aj.e2;
    const T s2 = sig * sig * rinv2;
    const T s6 = s2 * s2 * s2;
    // F / r = [Coulomb r^2 + 4 eps s6 (12 s6 - 6)] / r^2
    const T fs = keep ? fma(eps4 * s6, fma((T)12, s6, (T)-6), fcr) * rinv2 : (T)0;
    // explicit FMAs (never left to contraction), so the force and energy
    // variants of the kernel add every pair force with the same roundings
    fi.x = fma(-fs, dx, fi.x); fi.y = fma(-fs, dy, fi.y); fi.z = fma(-fs, dz, fi.z);
    fj.x = fma(fs, dx, fj.x);  fj.y = fma(fs, dy, fj.y);  fj.z = fma(fs, dz, fj.z);
    if (ENERGY) {
        // energies from correctly rounded arithmetic (energy steps only)
        const T re = t_sqrt_acc(r2);
        T erfc_e, ex_e;
        ewald_acc(re, r2, K, erfc_e, ex_e);
        const T vce = qq * erfc_e * t_rcp_acc(re);
        const T s2e = sig * sig * t_rcp_acc(r2);
        const T s6e = s2e * s2e * s2e;
        const T vlj = eps4 * fma(s6e, s6e, -s6e);
        elj += keep ? vlj : (T)0;
        ec += keep ? vce : (T)0;
    }
}

template <typename T>
__device__ __forceinline__ void red_jforce(const DevPtrs& P, int ja, int ii, T3<T> fj) {
    fj.x += __shfl_xor_sync(FULL, fj.x, 8);
    fj.y += __shfl_xor_sync(FULL, fj.y, 8);
    fj.z += __shfl_xor_sync(FULL, fj.z, 8);
    fj.x += __shfl_xor_sync(FULL, fj.x, 16);
    fj.y += __shfl_xor_sync(FULL, fj.y, 16);
    fj.z += __shfl_xor_sync(FULL, fj.z, 16);
    const T v = ii == 0 ? fj.x : (ii == 1 ? fj.y : fj.z);
    if (ii < 3 && v != (T)0) {
        long long* dst = ii == 0 ? P.fx : (ii == 1 ? P.fy : P.fz);
        add_fixed(dst + ja, (sizeof(T) == 4) ? to_fixed((float)v) : to_fixed_d((double)v));
    }
}

// i-forces: sum over the 8 lanes sharing ii, then lanes jj=0..2 write atom ii
// and lanes jj=3..5 write atom ii+4.
template <typename T>
__device__ __forceinline__ void red_iforce(const DevPtrs& P, int base_slot, int ii, int jj,
                                           T3<T> f0, T3<T> f1) {
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        f0.x += __shfl_xor_sync(FULL, f0.x, o);
        f0.y += __shfl_xor_sync(FULL, f0.y, o);
        f0.z += __shfl_xor_sync(FULL, f0.z, o);
        f1.x += __shfl_xor_sync(FULL, f1.x, o);
        f1.y += __shfl_xor_sync(FULL, f1.y, o);
        f1.z += __shfl_xor_sync(FULL, f1.z, o);
    }
    if (jj < 6) {
        const T3<T> f = jj < 3 ? f0 : f1;
        const int c = jj % 3;
        const T v = c == 0 ? f.x : (c == 1 ? f.y : f.z);
        if (v != (T)0) {
            long long* dst = c == 0 ? P.fx : (c == 1 ? P.fy : P.fz);
            const int a = base_slot + ii + (jj < 3 ? 0 : 4);
            add_fixed(dst + a, (sizeof(T) == 4) ? to_fixed((float)v) : to_fixed_d((double)v));
        }
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sums of 24 per-lane values over the warp by halving exchanges: at lane bit
// 4, 3, 2 each lane keeps the half of its values that matches its bit and adds
// the partner's copy of that half (12, 6, 3 shuffles), then bits 1 and 0 sum
// the remaining three in full. On return v[0] holds the sum of value
// 12 b4 + 6 b3 + 3 b2 + (lane & 3) for lane & 3 < 3 (the index is returned).
template <typename T>
__device__ __forceinline__ int warp_sum_24(T (&v)[24], int lane) {
    const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        const T keep = b4 ? v[j + 12] : v[j], give = b4 ? v[j] : v[j + 12];
        v[j] = keep + __shfl_xor_sync(FULL, give, 16);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const T keep = b3 ? v[j + 6] : v[j], give = b3 ? v[j] : v[j + 6];
        v[j] = keep + __shfl_xor_sync(FULL, give, 8);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const T keep = b2 ? v[j + 3] : v[j], give = b2 ? v[j] : v[j + 3];
        v[j] = keep + __shfl_xor_sync(FULL, give, 4);
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        v[j] += __shfl_xor_sync(FULL, v[j], 2);
        v[j] += __shfl_xor_sync(FULL, v[j], 1);
    }
    const int q = lane & 3;
    const T out = q == 1 ? v[1] : (q == 2 ? v[2] : v[0]);
    v[0] = out;
    return 12 * b4 + 6 * b3 + 3 * b2 + (q < 3 ? q : 0);
}

// ------------------------------------------------------------------ env rows
// Lane per j row: lane l of a warp takes row k0 + l of its item, loads the
// row's j atom once and evaluates it against the i atoms the row covers (all
// 8 for a full row, atoms 0-3 or 4-7 for a half row), read as broadcasts from
// the warp's copy of the i-cluster in shared memory. The j force stays in the
// lane and goes to the fixed-point accumulators once per row; the i forces
// stay in registers (8 atoms x 3) until the item ends and are then summed
// over the warp. A block of eight pairs per row gives every lane eight
// independent chains of arithmetic; a pair block no lane of the warp needs
// (a round of half rows of one kind) is skipped.
constexpr int ENV_WARPS_MAX = 8;

// one i atom in shared memory: x, y, z, q sqrt(ke), sigma/2, 2 sqrt(eps), -, -
template <typename T>
__device__ __forceinline__ Atom<T> ld_iatom(const T* p);
template <>
__device__ __forceinline__ Atom<float> ld_iatom<float>(const float* p) {
    const float4 a = reinterpret_cast<const float4*>(p)[0];
    const float4 b = reinterpret_cast<const float4*>(p)[1];
    return Atom<float>{a.x, a.y, a.z, a.w, b.x, b.y};
}
template <>
__device__ __forceinline__ Atom<double> ld_iatom<double>(const double* p) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    const double2 c = reinterpret_cast<const double2*>(p)[2];
    return Atom<double>{a.x, a.y, b.x, b.y, c.x, c.y};
}
template <typename T>
__device__ __forceinline__ void st_iatom(T* p, const Atom<T>& a) {
    p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.q; p[4] = a.sh; p[5] = a.e2;
    p[6] = (T)0; p[7] = (T)0;
}

// round kinds (warp-uniform): every lane a full row; every lane a row with
// only atoms 0-3 (LO) or only atoms 4-7 (HI) in range; anything else (mixed
// kinds, masked rows, idle lanes) with per-pair checks
enum : int { RM_FULL = 0, RM_LO = 1, RM_HI = 2, RM_MIXED = 3 };

// One row of a lane: its j atom (already shifted) against the i atoms of the
// active halves, minus the excluded ones (em) of a masked row; the j force
// goes to the accumulators.
template <typename T, bool ENERGY, int MODE>
__device__ __forceinline__ void env_row(const DevPtrs& P, const KC<T>& K, const T* s_ia, int ja,
                                        const Atom<T>& aj, bool act_lo, bool act_hi,
                                        unsigned int em, T3<T> (&fi)[CL], double& elj_d,
                                        double& ec_d) {
    T3<T> fj{(T)0, (T)0, (T)0};
    T elj = 0, ec = 0;
    constexpr int i0 = MODE == RM_HI ? 4 : 0, i1 = MODE == RM_LO ? 4 : CL;
#pragma unroll
    for (int ii = i0; ii < i1; ++ii) {
        if (MODE != RM_MIXED || ((ii < 4 ? act_lo : act_hi) && !((em >> ii) & 1u)))
            pair_env<T, ENERGY>(ld_iatom<T>(s_ia + ii * 8), aj, true, fi[ii], fj, elj, ec, K);
    }
    if (ENERGY) {
        elj_d += (double)elj;
        ec_d += (double)ec;
    }
    if (MODE != RM_MIXED || act_lo || act_hi) {
        const bool dbl = sizeof(T) == 8;
        if (fj.x != (T)0) add_fixed(P.fx + ja, dbl ? to_fixed_d((double)fj.x) : to_fixed((float)fj.x));
        if (fj.y != (T)0) add_fixed(P.fy + ja, dbl ? to_fixed_d((double)fj.y) : to_fixed((float)fj.y));
        if (fj.z != (T)0) add_fixed(P.fz + ja, dbl ? to_fixed_d((double)fj.z) : to_fixed((float)fj.z));
    }
}

// All rows of one item, 32 per round: row k < n_plain is plain row k (runs:
// full | atoms 0-3 only | atoms 4-7 only), row k >= n_plain masked row
// k - n_plain, so an item ends in one partly filled round. The next round's
// row word and j atom are loaded before the current round is computed (word,
// then atom: the loads depend on each other).
template <typename T, bool ENERGY>
__device__ __forceinline__ void env_rows(const DevPtrs& P, const KC<T>& K, const RepDev& R,
                                         const RowItem& I, const float4* sh, const T* s_ia,
                                         int lane, T3<T> (&fi)[CL], double& elj, double& ec) {
    const int n_full = I.cnt & 0xFFFF, n_lo_end = n_full + I.n_lo;
    const int n_plain = n_lo_end + I.n_hi, n = n_plain + (I.cnt >> 16);
    if (n <= 0) return;
    auto fetch = [&](int k, unsigned int& word, unsigned int& em) {
        const int kk = k < n ? k : n - 1;
        if (kk < n_plain) {
            word = P.rows[I.r_begin + (unsigned int)kk];
            em = 0u;
        } else {
            const int2 xr = P.xrows[I.x_begin + (kk - n_plain)];
            word = (unsigned int)xr.x;
            em = (unsigned int)xr.y;
        }
    };
    unsigned int word, em;
    fetch(lane, word, em);
    Atom<T> aj = load_atom<T>(P, (int)(word & ROW_SLOT_MASK), R, K);
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        unsigned int word_n = word, em_n = em;
        Atom<T> aj_n = aj;
        if (k0 + 32 < n) {   // warp-uniform
            fetch(k + 32, word_n, em_n);
            aj_n = load_atom<T>(P, (int)(word_n & ROW_SLOT_MASK), R, K);
        }
        // the j atom relative to the cluster's reference atom c, (x_j + u) - v
        // with (u, v) from the row's image code (see the table below)
        const int code = (int)(word >> ROW_SLOT_BITS);
        const float4 u = sh[code], v = sh[32 + code];
        Atom<T> a = aj;
        a.x = ((T)aj.x + (T)u.x) - (T)v.x;
        a.y = ((T)aj.y + (T)u.y) - (T)v.y;
        a.z = ((T)aj.z + (T)u.z) - (T)v.z;
        const int ja = (int)(word & ROW_SLOT_MASK);
        // the round's kind (warp-uniform)
        if (k0 + 32 <= n_full) {
            env_row<T, ENERGY, RM_FULL>(P, K, s_ia, ja, a, true, true, 0u, fi, elj, ec);
        } else if (k0 >= n_full && k0 + 32 <= n_lo_end) {
            env_row<T, ENERGY, RM_LO>(P, K, s_ia, ja, a, true, false, 0u, fi, elj, ec);
        } else if (k0 >= n_lo_end && k0 + 32 <= n_plain) {
            env_row<T, ENERGY, RM_HI>(P, K, s_ia, ja, a, false, true, 0u, fi, elj, ec);
        } else {
            const bool valid = k < n;
            const bool masked = k >= n_plain;
            const bool act_lo = valid && (masked || k < n_lo_end);
            const bool act_hi = valid && (masked || k < n_full || k >= n_lo_end);
            env_row<T, ENERGY, RM_MIXED>(P, K, s_ia, ja, a, act_lo, act_hi, em, fi, elj, ec);
        }
        word = word_n;
        em = em_n;
        aj = aj_n;
    }
}

template <typename T, bool ENERGY>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : (ENERGY ? 3 : 4)) k_env_rows(DevPtrs P) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    KC<T> K = make_kc<T>(P);
    __shared__ float4 s_ewtab[sizeof(T) == 4 ? EW_NT : 1];
    // per warp and image code: u (0-26) and v (32-58) of the shifted j atom
    // relative to the i-cluster's reference atom
    __shared__ float4 s_shift[ENV_WARPS_MAX][64];
    __shared__ __align__(16) T s_iat[ENV_WARPS_MAX][CL * 8];
    if constexpr (sizeof(T) == 4) {
        for (int i = threadIdx.x; i < EW_NT; i += blockDim.x) s_ewtab[i] = P.ewtab[i];
        __syncthreads();
        K.tab = s_ewtab;
    }
    float4* sh = s_shift[w];
    T* s_ia = s_iat[w];
    const int n_items = P.ritem_pref[P.R];
    // items are claimed up to four at a time (one claim per item serialised on
    // the counter: +0.5 ms per launch on the 1,152-window batch), fewer when
    // there are few items per warp
    const int chunk = max(1, min(4, n_items / ((int)(gridDim.x * (blockDim.x >> 5)) * 8)));
    int it_next = 0, it_end = 0;
    for (;;) {
        if (it_next >= it_end) {
            int c0 = 0;
            if (lane == 0) c0 = atomicAdd(&P.cnt->env_next, chunk);
            c0 = __shfl_sync(FULL, c0, 0);
            if (c0 >= n_items) break;
            it_next = c0;
            it_end = min(c0 + chunk, n_items);
        }
        const int it = it_next++;
        const RowItem I = row_item(P, it);
        const int rep = P.rep_of_cl[I.c];
        const RepDev& R = P.reps[rep];
        // image shifts of this replica's box, by code; the i-cluster's atoms
        // relative to its first atom (the reference c; same cluster: exact)
        // x_j + s - c for image shift s is evaluated as (x_j + u) - v with
        // u = s - c, v = 0 where s > 0 (then c lies near the box length, and
        // s - c is exact) and u = s, v = c otherwise (x_j + s is exact where
        // s < 0, x_j lying near the box length): no box-sized sum is rounded
        const float4 c = P.xq[I.c * CL];
        if (lane < 27) {
            const float sx = (float)(lane % 3 - 1) * R.box[0], sy = (float)((lane / 3) % 3 - 1) * R.box[1],
                        sz = (float)(lane / 9 - 1) * R.box[2];
            sh[lane] = make_float4(sx > 0.f ? sx - c.x : sx, sy > 0.f ? sy - c.y : sy,
                                   sz > 0.f ? sz - c.z : sz, 0.f);
            sh[32 + lane] = make_float4(sx > 0.f ? 0.f : c.x, sy > 0.f ? 0.f : c.y,
                                        sz > 0.f ? 0.f : c.z, 0.f);
        }
        if (lane < CL) {
            Atom<T> ai = load_atom<T>(P, I.c * CL + lane, R, K);
            ai.x -= (T)c.x;
            ai.y -= (T)c.y;
            ai.z -= (T)c.z;
            st_iatom<T>(s_ia + lane * 8, ai);
        }
        __syncwarp();
        T3<T> fi[CL];
#pragma unroll
        for (int ii = 0; ii < CL; ++ii) fi[ii] = T3<T>{(T)0, (T)0, (T)0};
        double elj = 0.0, ec = 0.0;
        env_rows<T, ENERGY>(P, K, R, I, sh, s_ia, lane, fi, elj, ec);
        // i forces: the 24 values 3 ii + c summed over the warp (transposed);
        // value v ends on the four lanes of group v / 3, and the lane with
        // lane % 4 == v % 3 < 3 writes it
        T v[3 * CL];
#pragma unroll
        for (int ii = 0; ii < CL; ++ii) {
            v[3 * ii] = fi[ii].x;
            v[3 * ii + 1] = fi[ii].y;
            v[3 * ii + 2] = fi[ii].z;
        }
        const int vi = warp_sum_24<T>(v, lane);
        if ((lane & 3) < 3 && v[0] != (T)0) {
            const int c = vi % 3;
            long long* d = c == 0 ? P.fx : (c == 1 ? P.fy : P.fz);
            add_fixed(d + I.c * CL + vi / 3,
                      (sizeof(T) == 4) ? to_fixed((float)v[0]) : to_fixed_d((double)v[0]));
        }
        if (ENERGY) {
            const double sl = warp_sum<double>(elj);
            const double sc = warp_sum<double>(ec);
            if (lane == 0) {
                if (!isfinite(sl) || !isfinite(sc)) set_err(P.cnt, ERRB_NONFINITE, rep);
                add_fixed(P.eacc + (size_t)rep * EA_N + EA_ENV_LJ, to_fixed_d(sl));
                add_fixed(P.eacc + (size_t)rep * EA_N + EA_ENV_C, to_fixed_d(sc));
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ ligand pair
template <typename T>
struct LigState {
    T lq, lv, A, dA, cs, dcs;
    bool soft;
};

template <typename T>
__device__ __forceinline__ void pair_lig(const Atom<T>& ai, const Atom<T>& aj, bool keep,
                                         const LigState<T>& S, T3<T>& fi, T3<T>& fj, T& elj,
                                         T& ec, T& dv, T& dq, const KC<T>& K) {
    const T dx = aj.x - ai.x, dy = aj.y - ai.y, dz = aj.z - ai.z;
    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
    keep = keep && (r2 < K.rc2);
    const T r = t_sqrt_acc(r2);
    const T rinv = t_rcp_acc(r);
    const T rinv2 = t_rcp_acc(r2);
    const T qq = ai.q * aj.q;
    T erfcv, ex;
    ewald_acc(r, r2, K, erfcv, ex);
    const T u1 = qq * erfcv * rinv;
    const T f1 = fma(qq * K.tbsp, ex, u1) * rinv2;
    const T sig = ai.sh + aj.sh;
    const T eps4 = ai.e2 * aj.e2;
    const T sig2 = sig * sig;
    const T sig6 = sig2 * sig2 * sig2;
    T ulj, flj, dudl;
    if (S.soft) {
        // Beutler: s6 = A sig^6 + r^6, A = alpha (1 - lambda)^p
        const T r4 = r2 * r2;
        const T s6 = fma(S.A, sig6, r4 * r2);
        const T inv = t_rcp_acc(s6);
        const T a = sig6 * inv;
        const T g = eps4 * fma(a, a, -a);
        const T dg = eps4 * fma((T)-2 * a, a, a) * inv;   // d g / d s6
        ulj = S.lv * g;
        flj = -S.lv * dg * (T)6 * r4;
        dudl = fma(S.lv * dg, S.dA * sig6, g);
    } else {
        const T s2 = sig2 * rinv2;
        const T s6 = s2 * s2 * s2;
        ulj = eps4 * fma(s6, s6, -s6);
        flj = eps4 * s6 * fma((T)12, s6, (T)-6) * rinv2;
        dudl = (T)0;
    }
    const T fs = keep ? fma(S.cs, f1, flj) : (T)0;
    fi.x = fma(-fs, dx, fi.x); fi.y = fma(-fs, dy, fi.y); fi.z = fma(-fs, dz, fi.z);
    fj.x = fma(fs, dx, fj.x);  fj.y = fma(fs, dy, fj.y);  fj.z = fma(fs, dz, fj.z);
    elj += keep ? ulj : (T)0;
    ec += keep ? S.cs * u1 : (T)0;
    dv += keep ? dudl : (T)0;
    dq += keep ? S.dcs * u1 : (T)0;
}

template <typename T>
__device__ __forceinline__ LigState<T> lig_state(const DevPtrs& P, const RepDev& R, int jlig);
template <>
__device__ __forceinline__ LigState<float> lig_state<float>(const DevPtrs& P, const RepDev& R,
                                                            int jlig) {
    LigState<float> S;
    S.lq = R.lam_q; S.lv = R.lam_v; S.A = R.sc_A; S.dA = R.sc_dA;
    const bool dec = P.ligand_mode == 1;
    S.soft = !(jlig && dec);
    if (!jlig) { S.cs = S.lq; S.dcs = 1.f; }
    else if (!dec) { S.cs = S.lq * S.lq; S.dcs = 2.f * S.lq; }
    else { S.cs = 1.f; S.dcs = 0.f; }
    return S;
}
template <>
__device__ __forceinline__ LigState<double> lig_state<double>(const DevPtrs& P, const RepDev& R,
                                                              int jlig) {
    LigState<double> S;
    S.lq = R.dlam_q; S.lv = R.dlam_v; S.A = R.dsc_A; S.dA = R.dsc_dA;
    const bool dec = P.ligand_mode == 1;
    S.soft = !(jlig && dec);
    if (!jlig) { S.cs = S.lq; S.dcs = 1.0; }
    else if (!dec) { S.cs = S.lq * S.lq; S.dcs = 2.0 * S.lq; }
    else { S.cs = 1.0; S.dcs = 0.0; }
    return S;
}

template <typename T, bool ENERGY>
__global__ void __launch_bounds__(128) k_lig(DevPtrs P) {
    const int lane = threadIdx.x & 31, jj = lane & 7, ii = lane >> 3;
    const KC<T> K = make_kc<T>(P);
    const int n_items = P.ilig_pref[P.R];
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&P.cnt->lig_next, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const Item I = P.items_lig[region_index(P.ilig_pref, P.ilig_base, P.R, it)];
        const RepDev& R = P.reps[I.rep];
        const int a0 = I.c0 * CL + ii;
        // coordinates relative to the cluster's first atom (see rel_img)
        const float4 c = P.xq[I.c0 * CL];
        Atom<T> ai0 = load_atom<T>(P, a0, R, K);
        Atom<T> ai1 = load_atom<T>(P, a0 + 4, R, K);
        ai0.x -= (T)c.x; ai0.y -= (T)c.y; ai0.z -= (T)c.z;
        ai1.x -= (T)c.x; ai1.y -= (T)c.y; ai1.z -= (T)c.z;
        T3<T> fi0{(T)0, (T)0, (T)0}, fi1{(T)0, (T)0, (T)0};
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const int ntot = I.e_cnt + I.x_cnt;
        for (int t = 0; t < ntot; ++t) {
            const bool xm = t >= I.e_cnt;
            const int k = xm ? I.x_begin + (t - I.e_cnt) : I.e_begin + t;
            const int2 e = xm ? P.xentries[k] : P.entries[k];
            const unsigned long long m = xm ? P.xmasks[(size_t)k * GMAX] : 0ull;
            const int jlig = entry_jlig(e.y);
            const LigState<T> S = lig_state<T>(P, R, jlig);
            float sx, sy, sz;
            entry_shift(e.y, R.box[0], R.box[1], R.box[2], sx, sy, sz);
            const int ja = e.x * CL + jj;
            Atom<T> aj = load_atom<T>(P, ja, R, K);
            aj.x = rel_img<T>((float)aj.x, sx, c.x);
            aj.y = rel_img<T>((float)aj.y, sy, c.y);
            aj.z = rel_img<T>((float)aj.z, sz, c.z);
            const bool k0 = !((m >> (ii * 8 + jj)) & 1ull);
            const bool k1 = !((m >> ((ii + 4) * 8 + jj)) & 1ull);
            T3<T> fj{(T)0, (T)0, (T)0};
            T elj = 0, ec = 0, dv = 0, dq = 0;
            pair_lig<T>(ai0, aj, k0, S, fi0, fj, elj, ec, dv, dq, K);
            pair_lig<T>(ai1, aj, k1, S, fi1, fj, elj, ec, dv, dq, K);
            red_jforce<T>(P, ja, ii, fj);
            if (ENERGY) {
                acc[jlig ? 1 : 0] += (double)elj;
                acc[jlig ? 3 : 2] += (double)ec;
                acc[4] += (double)dv;
                acc[5] += (double)dq;
            }
        }
        red_iforce<T>(P, I.c0 * CL, ii, jj, fi0, fi1);
        if (!ENERGY) continue;
        const int slot_map[6] = {EA_LIGENV_LJ, EA_LIGLIG_LJ, EA_LIGENV_C, EA_LIGLIG_C, EA_DUDLV,
                                 EA_DUDLQ};
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const double s = warp_sum<double>(acc[q]);
            if (lane == 0) {
                if (!isfinite(s)) set_err(P.cnt, ERRB_NONFINITE, I.rep);
                if (s != 0.0) add_fixed(P.eacc + (size_t)I.rep * EA_N + slot_map[q], to_fixed_d(s));
            }
        }
    }
}

// ------------------------------------------------------------------ u_kn
constexpr int UKN_WARPS = 2;

template <typename T>
__global__ void __launch_bounds__(UKN_WARPS * 32) k_lig_ukn(DevPtrs P) {
    __shared__ T s_acc[UKN_WARPS][KV_MAX][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, jj = lane & 7, ii = lane >> 3;
    const KC<T> K = make_kc<T>(P);
    const int n_items = P.ilig_pref[P.R];
    const bool dec = P.ligand_mode == 1;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&P.cnt->lig_next, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const Item I = P.items_lig[region_index(P.ilig_pref, P.ilig_base, P.R, it)];
        const RepDev& R = P.reps[I.rep];
        const int kv = R.kv;
        const float* kvl = P.kv_lam + R.sched * KV_MAX;
        const float* kva = P.kv_A + R.sched * KV_MAX;
        const double* kvld = P.kv_dlam + R.sched * KV_MAX;
        const double* kvad = P.kv_dA + R.sched * KV_MAX;
        for (int k = 0; k < kv; ++k) s_acc[w][k][lane] = (T)0;
        const int a0 = I.c0 * CL + ii;
        // coordinates relative to the cluster's first atom (see rel_img)
        const float4 c = P.xq[I.c0 * CL];
        Atom<T> ai[2] = {load_atom<T>(P, a0, R, K), load_atom<T>(P, a0 + 4, R, K)};
        for (int h = 0; h < 2; ++h) {
            ai[h].x -= (T)c.x; ai[h].y -= (T)c.y; ai[h].z -= (T)c.z;
        }
        double c_le = 0.0, c_ll = 0.0;
        const int ntot = I.e_cnt + I.x_cnt;
        for (int t = 0; t < ntot; ++t) {
            const bool xm = t >= I.e_cnt;
            const int k = xm ? I.x_begin + (t - I.e_cnt) : I.e_begin + t;
            const int2 e = xm ? P.xentries[k] : P.entries[k];
            const unsigned long long m = xm ? P.xmasks[(size_t)k * GMAX] : 0ull;
            const int jlig = entry_jlig(e.y);
            float sx, sy, sz;
            entry_shift(e.y, R.box[0], R.box[1], R.box[2], sx, sy, sz);
            const int ja = e.x * CL + jj;
            Atom<T> aj = load_atom<T>(P, ja, R, K);
            aj.x = rel_img<T>((float)aj.x, sx, c.x);
            aj.y = rel_img<T>((float)aj.y, sy, c.y);
            aj.z = rel_img<T>((float)aj.z, sz, c.z);
            const bool soft = !(jlig && dec);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool keep0 = !((m >> ((ii + 4 * h) * 8 + jj)) & 1ull);
                const T dx = aj.x - ai[h].x, dy = aj.y - ai[h].y, dz = aj.z - ai[h].z;
                const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const bool keep = keep0 && (r2 < K.rc2);
                if (keep) {
                    const T r = t_sqrt_acc(r2);
                    const T rinv = t_rcp_acc(r);
                    T erfcv, ex;
                    ewald_acc(r, r2, K, erfcv, ex);
                    const double u1 = (double)(ai[h].q * aj.q * erfcv * rinv);
                    if (!jlig) c_le += u1;
                    else if (!dec) c_ll += u1;
                    if (soft) {
                        const T sig = ai[h].sh + aj.sh;
                        const T eps4 = ai[h].e2 * aj.e2;
                        const T sig2 = sig * sig;
                        const T sig6 = sig2 * sig2 * sig2;
                        const T r6 = r2 * r2 * r2;
                        for (int q = 0; q < kv; ++q) {
                            const T lam = (sizeof(T) == 4) ? (T)kvl[q] : (T)kvld[q];
                            const T A = (sizeof(T) == 4) ? (T)kva[q] : (T)kvad[q];
                            const T a = sig6 * t_rcp_acc(fma(A, sig6, r6));
                            s_acc[w][q][lane] += lam * eps4 * fma(a, a, -a);
                        }
                    }
                }
            }
        }
        __syncwarp();
        for (int q = lane; q < kv; q += 32) {
            double s = 0.0;
            for (int l = 0; l < 32; ++l) s += (double)s_acc[w][q][l];
            if (!isfinite(s)) set_err(P.cnt, ERRB_NONFINITE, I.rep);
            if (s != 0.0) add_fixed(P.ukn_lj + (size_t)I.rep * KV_MAX + q, to_fixed_d(s));
        }
        const double sle = warp_sum<double>(c_le), sll = warp_sum<double>(c_ll);
        if (lane == 0) {
            if (sle != 0.0) add_fixed(P.ukn_c + (size_t)I.rep * 2 + 0, to_fixed_d(sle));
            if (sll != 0.0) add_fixed(P.ukn_c + (size_t)I.rep * 2 + 1, to_fixed_d(sll));
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ pair counting
// Environment pairs through the inner rows (the list the force kernel walks),
// in the force kernel's lane layout (lane per row, 32 rows per round, plain
// then masked rows); the item's computed pairs go to pair_cnt[2 R] in units
// of 32 for the lane efficiency: per round 32 lanes x 4 for each half block
// (atoms 0-3, 4-7) that some row of the round needs.
__global__ void __launch_bounds__(128) k_count_rows(DevPtrs P) {
    const int lane = threadIdx.x & 31;
    const int n_items = P.ritem_pref[P.R];
    const int stride = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += stride) {
        const RowItem I = row_item(P, it);
        const int rep = P.rep_of_cl[I.c];
        const RepDev& R = P.reps[rep];
        int cnt = 0;
        long long lanes = 0;
        const int n_full = I.cnt & 0xFFFF, n_lo_end = n_full + I.n_lo;
        const int n_plain = n_lo_end + I.n_hi, n = n_plain + (I.cnt >> 16);
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const bool valid = k < n, masked = k >= n_plain;
            const bool act_lo = valid && (masked || k < n_lo_end);
            const bool act_hi = valid && (masked || k < n_full || k >= n_lo_end);
            lanes += 128LL * ((__any_sync(0xffffffffu, act_lo) ? 1 : 0) +
                              (__any_sync(0xffffffffu, act_hi) ? 1 : 0));
            if (!valid) continue;
            unsigned int word, em = 0u;
            if (masked) {
                const int2 xr = P.xrows[I.x_begin + (k - n_plain)];
                word = (unsigned int)xr.x;
                em = (unsigned int)xr.y;
            } else {
                word = P.rows[I.r_begin + (unsigned int)k];
            }
            const int ja = (int)(word & ROW_SLOT_MASK), code = (int)(word >> ROW_SLOT_BITS);
            float4 xj = P.xq[ja];
            xj.x += (float)(code % 3 - 1) * R.box[0];
            xj.y += (float)((code / 3) % 3 - 1) * R.box[1];
            xj.z += (float)(code / 9 - 1) * R.box[2];
            const bool jreal = P.orig[ja] >= 0;
            for (int ii = 0; ii < CL; ++ii) {
                if (!(ii < 4 ? act_lo : act_hi) || ((em >> ii) & 1u)) continue;
                const int a = I.c * CL + ii;
                const float4 xi = P.xq[a];
                const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 < P.rc2 && jreal && P.orig[a] >= 0) {
                    ++cnt;
                    if (P.atom_cnt) {
                        atomicAdd(&P.atom_cnt[a], 1);
                        atomicAdd(&P.atom_cnt[ja], 1);
                    }
                }
            }
        }
        const int tot = warp_sum<int>(cnt);
        if (lane == 0 && tot)
            atomicAdd(reinterpret_cast<unsigned long long*>(P.pair_cnt + (size_t)rep * 2),
                      (unsigned long long)tot);
        if (lane == 0 && lanes)
            atomicAdd(reinterpret_cast<unsigned long long*>(P.pair_cnt + (size_t)P.R * 2),
                      (unsigned long long)(lanes / 32));
    }
}

// Ligand-involved pairs through the ligand list.
__global__ void __launch_bounds__(128) k_count_lig(DevPtrs P) {
    const int lane = threadIdx.x & 31, jj = lane & 7, ii = lane >> 3;
    const int n_items = P.ilig_pref[P.R];
    const int stride = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += stride) {
        const Item I = P.items_lig[region_index(P.ilig_pref, P.ilig_base, P.R, it)];
        const RepDev& R = P.reps[I.rep];
        int cnt = 0;
        const int ntot = I.e_cnt + I.x_cnt;
        for (int t = 0; t < ntot; ++t) {
            const bool xm = t >= I.e_cnt;
            const int k = xm ? I.x_begin + (t - I.e_cnt) : I.e_begin + t;
            const int2 e = xm ? P.xentries[k] : P.entries[k];
            float sx, sy, sz;
            entry_shift(e.y, R.box[0], R.box[1], R.box[2], sx, sy, sz);
            const int ja = e.x * CL + jj;
            float4 xj = P.xq[ja];
            xj.x += sx; xj.y += sy; xj.z += sz;
            const bool jreal = P.orig[ja] >= 0;
            for (int g = 0; g < I.ng; ++g) {
                const unsigned long long m = xm ? P.xmasks[(size_t)k * GMAX + g] : 0ull;
                for (int h = 0; h < 2; ++h) {
                    if (!entry_half(e.y, g, h)) continue;
                    const int a = (I.c0 + g) * CL + ii + 4 * h;
                    const float4 xi = P.xq[a];
                    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const bool keep = !((m >> ((ii + 4 * h) * 8 + jj)) & 1ull) && r2 < P.rc2 &&
                                      jreal && P.orig[a] >= 0;
                    if (keep) {
                        ++cnt;
                        if (P.atom_cnt) {
                            atomicAdd(&P.atom_cnt[a], 1);
                            atomicAdd(&P.atom_cnt[ja], 1);
                        }
                    }
                }
            }
        }
        const int tot = warp_sum<int>(cnt);
        if (lane == 0 && tot)
            atomicAdd(reinterpret_cast<unsigned long long*>(P.pair_cnt + (size_t)I.rep * 2 + 1),
                      (unsigned long long)tot);
    }
}

}  // namespace

void launch_env_forces(const DevPtrs& P, cudaStream_t s, bool energy, int precision, int grid,
                       int block) {
    if (precision == 1) k_env_rows<double, true><<<grid, block, 0, s>>>(P);
    else if (energy) k_env_rows<float, true><<<grid, block, 0, s>>>(P);
    else k_env_rows<float, false><<<grid, block, 0, s>>>(P);
}

int env_kernel_occupancy(int block, int precision, bool energy) {
    int nb = 0;
    if (precision == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<double, true>, block, 0);
    else if (energy)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<float, true>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<float, false>, block, 0);
    return nb;
}

void launch_lig_forces(const DevPtrs& P, cudaStream_t s, int precision, int grid, int block,
                       bool energy) {
    // force steps skip the energy sums (FP64 adds: the FP64 pipe bounds them)
    if (precision == 1) {
        if (energy) k_lig<double, true><<<grid, block, 0, s>>>(P);
        else k_lig<double, false><<<grid, block, 0, s>>>(P);
    } else {
        if (energy) k_lig<float, true><<<grid, block, 0, s>>>(P);
        else k_lig<float, false><<<grid, block, 0, s>>>(P);
    }
}

void launch_lig_ukn(const DevPtrs& P, cudaStream_t s, int grid, int precision) {
    if (precision == 1) k_lig_ukn<double><<<grid, UKN_WARPS * 32, 0, s>>>(P);
    else k_lig_ukn<float><<<grid, UKN_WARPS * 32, 0, s>>>(P);
}

void launch_count_pairs(const DevPtrs& P, cudaStream_t s, int grid, int block) {
    k_count_rows<<<grid, block, 0, s>>>(P);
    k_count_lig<<<grid, block, 0, s>>>(P);
}

}  // namespace abfe
