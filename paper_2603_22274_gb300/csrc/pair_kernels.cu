// Cluster-pair nonbonded kernels.
//
// Warp layout (both kernels): lane = jj + 8*ii, jj = j-atom of the current
// j cluster (0..7), ii = 0..3; the lane owns i-atoms ii and ii+4 of every
// i-cluster of its work item. Per j-cluster entry a lane evaluates two pairs per
// active i-cluster, the j-force is summed over the four lanes sharing jj with two
// xor-shuffles and added to the 64-bit fixed-point accumulators by three lanes
// at once; i-forces stay in registers until the item ends.
//
// * k_env: environment-environment pairs (lambda independent): plain 12-6 LJ
//   with Lorentz-Berthelot mixing plus real-space Ewald Coulomb, hard cutoff.
//   FP32 forces: the Coulomb force is qq G(r^2) / r^3 with G from a quadratic
//   table in r^2 held in shared memory (ewald_G); FP32 energies (energy steps
//   only) use correctly rounded arithmetic and erfcf/expf; FP64 uses erfc/exp.
// * k_lig: ligand-involved pairs at the replica's own state: Beutler softcore
//   LJ, lambda_q-scaled charges, dU/dlambda_v and dU/dlambda_q; pair arithmetic
//   in the kernel's precision, sums in FP64.
// * k_lig_ukn: the same pairs at every distinct lambda_v of the replica's
//   schedule, plus the unit-charge Coulomb sums, for the u_kn row.
// * k_count: in-cutoff pair counts through the list (list parity checks).
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
__device__ __forceinline__ Atom<T> load_atom(const DevPtrs& P, int slot, int sys_atom_off,
                                             const KC<T>& K);
template <>
__device__ __forceinline__ Atom<float> load_atom<float>(const DevPtrs& P, int slot, int,
                                                        const KC<float>&) {
    const float4 x = P.xq[slot];
    const float2 s = P.se[slot];
    return Atom<float>{x.x, x.y, x.z, x.w, s.x, s.y};
}
template <>
__device__ __forceinline__ Atom<double> load_atom<double>(const DevPtrs& P, int slot,
                                                          int sys_atom_off, const KC<double>& K) {
    const float4 x = P.xq[slot];
    const int o = P.orig[slot];
    Atom<double> a{(double)x.x, (double)x.y, (double)x.z, 0.0, 0.0, 0.0};
    if (o >= 0) {
        const dbl4 p = P.sys_prmd[sys_atom_off + o];
        a.q = p.x * K.dke_sqrt;
        a.sh = 0.5 * p.y;
        a.e2 = 2.0 * sqrt(p.z);
    }
    return a;
}

__device__ __forceinline__ float t_rsqrt(float x) { return rsqrt_fast(x); }
__device__ __forceinline__ double t_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float t_rcp(float x) { return rcp_fast(x); }
__device__ __forceinline__ double t_rcp(double x) { return 1.0 / x; }

// erfc(beta r) and exp(-beta^2 r^2)
__device__ __forceinline__ void ewald(float r, float r2, const KC<float>& K, float& erfcv,
                                      float& ex) {
    ex = ex2_fast(r2 * K.nb2l2e);
    erfcv = erfcx_fit(r * K.beta) * ex;
}
__device__ __forceinline__ void ewald(double r, double r2, const KC<double>& K, double& erfcv,
                                      double& ex) {
    ex = exp(-K.beta * K.beta * r2);
    erfcv = erfc(K.beta * r);
}

// G(r^2) from the shared-memory table: the nearest grid point j = round(t),
// t = r^2 / h (clamped to the table), and the centred quadratic in f = t - j.
// Adding 1.5 * 2^23 leaves round(t) in the low mantissa bits (t < 2^22), so no
// conversion instruction is needed.
__device__ __forceinline__ float ewald_G(float r2, const float4* tab, float inv_h) {
    const float t = fminf(r2 * inv_h, (float)(EW_NT - 1));
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

template <typename T>
__device__ __forceinline__ void shift_of(int y, const RepDev& R, T& sx, T& sy, T& sz) {
    float fx, fy, fz;
    entry_shift(y, R.box[0], R.box[1], R.box[2], fx, fy, fz);
    sx = (T)fx; sy = (T)fy; sz = (T)fz;
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
    T fc;
    if constexpr (sizeof(T) == 4) {
        // Coulomb force qq G(r^2) / r^3 from the table
        fc = qq * ewald_G(r2, K.tab, K.inv_h) * rinv * rinv2;
    } else {
        const T r = r2 * rinv;
        T erfcv, ex;
        ewald(r, r2, K, erfcv, ex);
        const T vc = qq * erfcv * rinv;
        fc = fma(qq * K.tbsp, ex, vc) * rinv2;
    }
    const T sig = ai.sh + aj.sh;
    const T eps4 = ai.e2 * aj.e2;
    const T s2 = sig * sig * rinv2;
    const T s6 = s2 * s2 * s2;
    const T flj = eps4 * s6 * fma((T)12, s6, (T)-6) * rinv2;
    const T fs = keep ? (fc + flj) : (T)0;
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

template <typename T, int G, bool ENERGY, bool XM>
__device__ __forceinline__ void env_entry(const DevPtrs& P, const KC<T>& K, const RepDev& R,
                                          int2 e, const unsigned long long* m, int ii, int jj,
                                          const Atom<T> (&ai0)[G], const Atom<T> (&ai1)[G],
                                          T3<T> (&fi0)[G], T3<T> (&fi1)[G], double& elj_d,
                                          double& ec_d) {
    const int jc = e.x, y = e.y;
    const int ja = jc * CL + jj;
    Atom<T> aj = load_atom<T>(P, ja, R.sys_atom_off, K);
    if ((y & ENTRY_SHIFT_BITS) != ENTRY_NOSHIFT) {  // periodic image (warp-uniform)
        T sx, sy, sz;
        shift_of<T>(y, R, sx, sy, sz);
        aj.x += sx; aj.y += sy; aj.z += sz;
    }
    T3<T> fj{(T)0, (T)0, (T)0};
    T elj = 0, ec = 0;  // this entry's energy (at most 2G pairs), then added in FP64
#pragma unroll
    for (int g = 0; g < G; ++g) {
        // each half tile (rows ii or ii+4 of i-cluster g) is a warp-uniform branch
        if (entry_half(y, g, 0)) {
            const bool k0 = XM ? !((m[g] >> (ii * 8 + jj)) & 1ull) : true;
            pair_env<T, ENERGY>(ai0[g], aj, k0, fi0[g], fj, elj, ec, K);
        }
        if (entry_half(y, g, 1)) {
            const bool k1 = XM ? !((m[g] >> ((ii + 4) * 8 + jj)) & 1ull) : true;
            pair_env<T, ENERGY>(ai1[g], aj, k1, fi1[g], fj, elj, ec, K);
        }
    }
    if (ENERGY) {
        elj_d += (double)elj;
        ec_d += (double)ec;
    }
    red_jforce<T>(P, ja, ii, fj);
}

template <typename T, int G, bool ENERGY>
__global__ void __launch_bounds__(256, (G == 4 || sizeof(T) == 8) ? 2 : 4) k_env(DevPtrs P) {
    const int lane = threadIdx.x & 31, jj = lane & 7, ii = lane >> 3;
    KC<T> K = make_kc<T>(P);
    __shared__ float4 s_ewtab[sizeof(T) == 4 ? EW_NT : 1];
    if constexpr (sizeof(T) == 4) {
        for (int i = threadIdx.x; i < EW_NT; i += blockDim.x) s_ewtab[i] = P.ewtab[i];
        __syncthreads();
        K.tab = s_ewtab;
    }
    const int n_items = min(*(volatile int*)&P.cnt->n_items_env, P.cap_items_env);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&P.cnt->env_next, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const Item I = P.items_env[it];
        const RepDev& R = P.reps[I.rep];
        Atom<T> ai0[G], ai1[G];
        T3<T> fi0[G], fi1[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            fi0[g] = T3<T>{(T)0, (T)0, (T)0};
            fi1[g] = T3<T>{(T)0, (T)0, (T)0};
            if (g < I.ng) {
                const int a = (I.c0 + g) * CL + ii;
                ai0[g] = load_atom<T>(P, a, R.sys_atom_off, K);
                ai1[g] = load_atom<T>(P, a + 4, R.sys_atom_off, K);
            } else {
                ai0[g] = Atom<T>{(T)0, (T)0, (T)0, (T)0, (T)0, (T)0};
                ai1[g] = ai0[g];
            }
        }
        double elj = 0.0, ec = 0.0;
        const int e_end = I.e_begin + I.e_cnt;
        for (int k = I.e_begin; k < e_end; ++k) {
            const int2 e = P.entries[k];
            env_entry<T, G, ENERGY, false>(P, K, R, e, nullptr, ii, jj, ai0, ai1, fi0, fi1, elj, ec);
        }
        const int x_end = I.x_begin + I.x_cnt;
        for (int k = I.x_begin; k < x_end; ++k) {
            const int2 e = P.xentries[k];
            unsigned long long m[G];
#pragma unroll
            for (int g = 0; g < G; ++g) m[g] = P.xmasks[(size_t)k * GMAX + g];
            env_entry<T, G, ENERGY, true>(P, K, R, e, m, ii, jj, ai0, ai1, fi0, fi1, elj, ec);
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
            if (g < I.ng) red_iforce<T>(P, (I.c0 + g) * CL, ii, jj, fi0[g], fi1[g]);
        if (ENERGY) {
            const double sl = warp_sum<double>(elj);
            const double sc = warp_sum<double>(ec);
            if (lane == 0) {
                if (!isfinite(sl) || !isfinite(sc)) set_err(P.cnt, ERRB_NONFINITE, I.rep);
                add_fixed(P.eacc + (size_t)I.rep * EA_N + EA_ENV_LJ, to_fixed_d(sl));
                add_fixed(P.eacc + (size_t)I.rep * EA_N + EA_ENV_C, to_fixed_d(sc));
            }
        }
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

template <typename T>
__global__ void __launch_bounds__(128) k_lig(DevPtrs P) {
    const int lane = threadIdx.x & 31, jj = lane & 7, ii = lane >> 3;
    const KC<T> K = make_kc<T>(P);
    const int n_items = min(*(volatile int*)&P.cnt->n_items_lig, P.cap_items_lig);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&P.cnt->lig_next, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const Item I = P.items_lig[it];
        const RepDev& R = P.reps[I.rep];
        const int a0 = I.c0 * CL + ii;
        const Atom<T> ai0 = load_atom<T>(P, a0, R.sys_atom_off, K);
        const Atom<T> ai1 = load_atom<T>(P, a0 + 4, R.sys_atom_off, K);
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
            T sx, sy, sz;
            shift_of<T>(e.y, R, sx, sy, sz);
            const int ja = e.x * CL + jj;
            Atom<T> aj = load_atom<T>(P, ja, R.sys_atom_off, K);
            aj.x += sx; aj.y += sy; aj.z += sz;
            const bool k0 = !((m >> (ii * 8 + jj)) & 1ull);
            const bool k1 = !((m >> ((ii + 4) * 8 + jj)) & 1ull);
            T3<T> fj{(T)0, (T)0, (T)0};
            T elj = 0, ec = 0, dv = 0, dq = 0;
            pair_lig<T>(ai0, aj, k0, S, fi0, fj, elj, ec, dv, dq, K);
            pair_lig<T>(ai1, aj, k1, S, fi1, fj, elj, ec, dv, dq, K);
            red_jforce<T>(P, ja, ii, fj);
            acc[jlig ? 1 : 0] += (double)elj;
            acc[jlig ? 3 : 2] += (double)ec;
            acc[4] += (double)dv;
            acc[5] += (double)dq;
        }
        red_iforce<T>(P, I.c0 * CL, ii, jj, fi0, fi1);
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
    const int n_items = min(*(volatile int*)&P.cnt->n_items_lig, P.cap_items_lig);
    const bool dec = P.ligand_mode == 1;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&P.cnt->lig_next, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const Item I = P.items_lig[it];
        const RepDev& R = P.reps[I.rep];
        const int kv = R.kv;
        const float* kvl = P.kv_lam + R.sched * KV_MAX;
        const float* kva = P.kv_A + R.sched * KV_MAX;
        const double* kvld = P.kv_dlam + R.sched * KV_MAX;
        const double* kvad = P.kv_dA + R.sched * KV_MAX;
        for (int k = 0; k < kv; ++k) s_acc[w][k][lane] = (T)0;
        const int a0 = I.c0 * CL + ii;
        const Atom<T> ai[2] = {load_atom<T>(P, a0, R.sys_atom_off, K),
                               load_atom<T>(P, a0 + 4, R.sys_atom_off, K)};
        double c_le = 0.0, c_ll = 0.0;
        const int ntot = I.e_cnt + I.x_cnt;
        for (int t = 0; t < ntot; ++t) {
            const bool xm = t >= I.e_cnt;
            const int k = xm ? I.x_begin + (t - I.e_cnt) : I.e_begin + t;
            const int2 e = xm ? P.xentries[k] : P.entries[k];
            const unsigned long long m = xm ? P.xmasks[(size_t)k * GMAX] : 0ull;
            const int jlig = entry_jlig(e.y);
            T sx, sy, sz;
            shift_of<T>(e.y, R, sx, sy, sz);
            const int ja = e.x * CL + jj;
            Atom<T> aj = load_atom<T>(P, ja, R.sys_atom_off, K);
            aj.x += sx; aj.y += sy; aj.z += sz;
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
template <bool LIG>
__global__ void __launch_bounds__(128) k_count(DevPtrs P) {
    const int lane = threadIdx.x & 31, jj = lane & 7, ii = lane >> 3;
    const int n_items = min(*(volatile int*)(LIG ? &P.cnt->n_items_lig : &P.cnt->n_items_env),
                            LIG ? P.cap_items_lig : P.cap_items_env);
    const int stride = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += stride) {
        const Item I = LIG ? P.items_lig[it] : P.items_env[it];
        const RepDev& R = P.reps[I.rep];
        int cnt = 0, halves = 0;
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
                    ++halves;
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
            atomicAdd(reinterpret_cast<unsigned long long*>(P.pair_cnt + (size_t)I.rep * 2 + (LIG ? 1 : 0)),
                      (unsigned long long)tot);
        // every lane walked the same entries: lane 0's count is the item's half tiles
        if (!LIG && lane == 0 && halves)
            atomicAdd(reinterpret_cast<unsigned long long*>(P.pair_cnt + (size_t)P.R * 2),
                      (unsigned long long)halves);
    }
}

}  // namespace

void launch_env_forces(const DevPtrs& P, cudaStream_t s, bool energy, int precision, int grid,
                       int block) {
    if (precision == 1) {
        k_env<double, 1, true><<<grid, block, 0, s>>>(P);
        return;
    }
    switch (P.group) {
        case 1:
            if (energy) k_env<float, 1, true><<<grid, block, 0, s>>>(P);
            else k_env<float, 1, false><<<grid, block, 0, s>>>(P);
            break;
        case 2:
            if (energy) k_env<float, 2, true><<<grid, block, 0, s>>>(P);
            else k_env<float, 2, false><<<grid, block, 0, s>>>(P);
            break;
        default:
            if (energy) k_env<float, 4, true><<<grid, block, 0, s>>>(P);
            else k_env<float, 4, false><<<grid, block, 0, s>>>(P);
            break;
    }
}

int env_kernel_occupancy(int group, int block, int precision, bool energy) {
    int nb = 0;
    if (precision == 1) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env<double, 1, true>, block, 0);
        return nb;
    }
    switch (group) {
        case 1:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &nb, energy ? k_env<float, 1, true> : k_env<float, 1, false>, block, 0);
            break;
        case 2:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &nb, energy ? k_env<float, 2, true> : k_env<float, 2, false>, block, 0);
            break;
        default:
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &nb, energy ? k_env<float, 4, true> : k_env<float, 4, false>, block, 0);
            break;
    }
    return nb;
}

void launch_lig_forces(const DevPtrs& P, cudaStream_t s, int precision, int grid, int block) {
    if (precision == 1) k_lig<double><<<grid, block, 0, s>>>(P);
    else k_lig<float><<<grid, block, 0, s>>>(P);
}

void launch_lig_ukn(const DevPtrs& P, cudaStream_t s, int grid, int precision) {
    if (precision == 1) k_lig_ukn<double><<<grid, UKN_WARPS * 32, 0, s>>>(P);
    else k_lig_ukn<float><<<grid, UKN_WARPS * 32, 0, s>>>(P);
}

void launch_count_pairs(const DevPtrs& P, cudaStream_t s, int grid, int block) {
    k_count<false><<<grid, block, 0, s>>>(P);
    k_count<true><<<grid, block, 0, s>>>(P);
}

}  // namespace abfe
