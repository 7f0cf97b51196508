// Nonbonded pair kernels.
//
// * k_env_rows: environment-environment pairs (lambda independent): plain
//   12-6 LJ with Lorentz-Berthelot mixing plus real-space Ewald Coulomb, hard
//   cutoff, over the inner list of j rows. A warp owns one i-cluster (8 atoms)
//   and walks its rows eight at a time: lane = q + 4 slot (q = 0..3, slot =
//   0..7) evaluates i atoms q and q+4 against the j atom of row `slot`, so one
//   j load serves two pairs; the j force is summed over the four lanes of the
//   slot by a transposed shuffle reduction (three shuffles leave x, y and z on
//   three lanes) and added to the 64-bit fixed-point accumulators; i forces
//   stay in registers until the item ends. FP32 forces: the Coulomb force is
//   qq G(r^2) / r^3 with G from a quadratic table in r^2 held in shared memory
//   (ewald_G); FP32 energies (energy steps only) use correctly rounded
//   arithmetic and erfcf/expf; FP64 uses erfc/exp.
// * k_lig: ligand-involved pairs at the replica's own state (outer list, 4x8
//   half tiles: lane = jj + 8 ii): Beutler softcore LJ, lambda_q-scaled
//   charges, dU/dlambda_v and dU/dlambda_q; pair arithmetic in the kernel's
//   precision, sums in FP64.
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
    T fcr;  // Coulomb force times r^2
    if constexpr (sizeof(T) == 4) {
        // Coulomb force qq G(r^2) / r^3 from the table
        fcr = qq * ewald_G(r2, K.tab, K.inv_h) * rinv;
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

// j force of one row, summed over the four lanes q = 0..3 that share its j atom:
// a transposed reduction (lanes keep different components at each level)
// leaves the x sum on q = 0, y on q = 1 and z on q = 2 and 3, which add it to
// the fixed-point accumulators.
template <typename T>
__device__ __forceinline__ void red_row(const DevPtrs& P, long long* dst, int ja, int q,
                                        T3<T> f) {
    const bool b0 = q & 1, b1 = (q >> 1) & 1;
    const T r1 = __shfl_xor_sync(FULL, b0 ? f.x : f.y, 1);
    const T a = (b0 ? f.y : f.x) + r1;
    f.z += __shfl_xor_sync(FULL, f.z, 1);
    const T r2 = __shfl_xor_sync(FULL, b1 ? a : f.z, 2);
    const T v = (b1 ? f.z : a) + r2;
    if (q < 3 && v != (T)0)
        add_fixed(dst + ja, (sizeof(T) == 4) ? to_fixed((float)v) : to_fixed_d((double)v));
}

// Packed FP32 pairs (sm_100 family f32x2 instructions): the two pairs a lane
// evaluates per round share the j atom, so their arithmetic runs as one packed
// stream, value for i atom q in the low and for q+4 in the high half.
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(u64 r, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// the lane's two i atoms, packed
struct AtomPair {
    u64 x, y, z, q, sh, e2;
};
__device__ __forceinline__ AtomPair pack_atoms(const Atom<float>& a, const Atom<float>& b) {
    return AtomPair{pk2(a.x, b.x), pk2(a.y, b.y), pk2(a.z, b.z),
                    pk2(a.q, b.q), pk2(a.sh, b.sh), pk2(a.e2, b.e2)};
}

// pair_env's force arithmetic for the lane's two pairs at once; i forces
// accumulate packed, the j force returns summed over the two pairs
__device__ __forceinline__ void pair_env2(const AtomPair& ai, const Atom<float>& aj, bool k0, bool k1,
                                          u64& fx, u64& fy, u64& fz, T3<float>& fj,
                                          const KC<float>& K) {
    const u64 dx = sub2(pk2(aj.x, aj.x), ai.x);
    const u64 dy = sub2(pk2(aj.y, aj.y), ai.y);
    const u64 dz = sub2(pk2(aj.z, aj.z), ai.z);
    const u64 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
    float r2a, r2b;
    up2(r2, r2a, r2b);
    const bool ka = k0 && (r2a < K.rc2), kb = k1 && (r2b < K.rc2);
    const u64 rinv = pk2(rsqrt_fast(r2a), rsqrt_fast(r2b));
    const u64 rinv2 = mul2(rinv, rinv);
    const u64 qq = mul2(ai.q, pk2(aj.q, aj.q));
    const u64 g = pk2(ewald_G(r2a, K.tab, K.inv_h), ewald_G(r2b, K.tab, K.inv_h));
    const u64 fcr = mul2(mul2(qq, g), rinv);
    const u64 sig = add2(ai.sh, pk2(aj.sh, aj.sh));
    const u64 eps4 = mul2(ai.e2, pk2(aj.e2, aj.e2));
    const u64 s2 = mul2(mul2(sig, sig), rinv2);
    const u64 s6 = mul2(mul2(s2, s2), s2);
    const u64 f = mul2(fma2(mul2(eps4, s6), fma2(pk2(12.f, 12.f), s6, pk2(-6.f, -6.f)), fcr), rinv2);
    float fa, fb;
    up2(f, fa, fb);
    const u64 fs = pk2(ka ? fa : 0.f, kb ? fb : 0.f);
    const u64 px = mul2(fs, dx), py = mul2(fs, dy), pz = mul2(fs, dz);
    fx = sub2(fx, px);
    fy = sub2(fy, py);
    fz = sub2(fz, pz);
    float a, b;
    up2(px, a, b);
    fj.x = a + b;
    up2(py, a, b);
    fj.y = a + b;
    up2(pz, a, b);
    fj.z = a + b;
}

constexpr int ROWS_PER_ROUND = 8;
constexpr int ROW_WARPS_MAX = 8;

// The i-side state of a lane: its two atoms and forces, scalar or packed.
template <typename T, bool PACK>
struct ILane {
    Atom<T> a0, a1;
    T3<T> f0, f1;
    AtomPair ap;       // PACK: the two atoms packed
    u64 fx, fy, fz;    // PACK: the two forces packed
};

template <typename T, bool ENERGY, bool MASKED, bool PACK>
__device__ __forceinline__ void row_round(const DevPtrs& P, const KC<T>& K, int ja, Atom<T> aj,
                                          unsigned int code, unsigned int em, bool valid,
                                          const float4* sh, int q, long long* dst,
                                          ILane<T, PACK>& L, double& elj_d, double& ec_d) {
    const float4 s = sh[code];
    aj.x += (T)s.x; aj.y += (T)s.y; aj.z += (T)s.z;
    const bool k0 = MASKED ? valid && !((em >> q) & 1u) : valid;
    const bool k1 = MASKED ? valid && !((em >> (q + 4)) & 1u) : valid;
    T3<T> fj{(T)0, (T)0, (T)0};
    if constexpr (PACK) {
        pair_env2(L.ap, aj, k0, k1, L.fx, L.fy, L.fz, fj, K);
    } else {
        T elj = 0, ec = 0;
        pair_env<T, ENERGY>(L.a0, aj, k0, L.f0, fj, elj, ec, K);
        pair_env<T, ENERGY>(L.a1, aj, k1, L.f1, fj, elj, ec, K);
        if (ENERGY) {
            elj_d += (double)elj;
            ec_d += (double)ec;
        }
    }
    red_row<T>(P, dst, ja, q, fj);
}

// Rows [b, e) of one item, eight per round; the next round's row word and j atom
// are loaded before the current round is computed (the loads of a round depend
// on each other: word, then atom).
template <typename T, bool ENERGY, bool MASKED, bool PACK>
__device__ __forceinline__ void row_loop(const DevPtrs& P, const KC<T>& K, const RepDev& R,
                                         unsigned int b, unsigned int e, int slot,
                                         const float4* sh, int q, long long* dst,
                                         ILane<T, PACK>& L, double& elj, double& ec) {
    if (b >= e) return;
    auto fetch = [&](unsigned int k, unsigned int& word, unsigned int& em) {
        const unsigned int kk = k < e ? k : e - 1u;
        if (MASKED) {
            const int2 xr = P.xrows[kk];
            word = (unsigned int)xr.x;
            em = (unsigned int)xr.y;
        } else {
            word = P.rows[kk];
            em = 0u;
        }
    };
    unsigned int word, em;
    fetch(b + slot, word, em);
    Atom<T> aj = load_atom<T>(P, (int)(word & ROW_SLOT_MASK), R, K);
    for (unsigned int k0 = b; k0 < e; k0 += ROWS_PER_ROUND) {
        const unsigned int kn = k0 + ROWS_PER_ROUND;
        unsigned int word_n = word, em_n = em;
        Atom<T> aj_n = aj;
        if (kn < e) {   // warp-uniform
            fetch(kn + slot, word_n, em_n);
            aj_n = load_atom<T>(P, (int)(word_n & ROW_SLOT_MASK), R, K);
        }
        row_round<T, ENERGY, MASKED, PACK>(P, K, (int)(word & ROW_SLOT_MASK), aj,
                                           word >> ROW_SLOT_BITS, em, k0 + slot < e, sh, q, dst,
                                           L, elj, ec);
        word = word_n;
        em = em_n;
        aj = aj_n;
    }
}

template <typename T, bool ENERGY, bool PACK>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 4) k_env_rows(DevPtrs P) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = lane & 3, slot = lane >> 2;
    KC<T> K = make_kc<T>(P);
    __shared__ float4 s_ewtab[sizeof(T) == 4 ? EW_NT : 1];
    __shared__ float4 s_shift[ROW_WARPS_MAX][28];
    if constexpr (sizeof(T) == 4) {
        for (int i = threadIdx.x; i < EW_NT; i += blockDim.x) s_ewtab[i] = P.ewtab[i];
        __syncthreads();
        K.tab = s_ewtab;
    }
    float4* sh = s_shift[w];
    long long* dst = q == 0 ? P.fx : (q == 1 ? P.fy : P.fz);
    const int n_items = min(*(volatile int*)&P.cnt->n_ritems, P.cap_ritems);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&P.cnt->env_next, 1);
        it = __shfl_sync(FULL, it, 0);
        if (it >= n_items) break;
        const RowItem I = P.ritems[it];
        const int rep = P.rep_of_cl[I.c];
        const RepDev& R = P.reps[rep];
        const int r_cnt = I.cnt & 0xFFFF, x_cnt = I.cnt >> 16;
        // image shifts of this replica's box, by code
        if (lane < 27)
            sh[lane] = make_float4((float)(lane % 3 - 1) * R.box[0],
                                   (float)((lane / 3) % 3 - 1) * R.box[1],
                                   (float)(lane / 9 - 1) * R.box[2], 0.f);
        __syncwarp();
        ILane<T, PACK> L;
        L.a0 = load_atom<T>(P, I.c * CL + q, R, K);
        L.a1 = load_atom<T>(P, I.c * CL + q + 4, R, K);
        L.f0 = T3<T>{(T)0, (T)0, (T)0};
        L.f1 = T3<T>{(T)0, (T)0, (T)0};
        if constexpr (PACK) {
            L.ap = pack_atoms(L.a0, L.a1);
            L.fx = L.fy = L.fz = pk2(0.f, 0.f);
        }
        double elj = 0.0, ec = 0.0;
        row_loop<T, ENERGY, false, PACK>(P, K, R, I.r_begin, I.r_begin + (unsigned int)r_cnt, slot,
                                         sh, q, dst, L, elj, ec);
        row_loop<T, ENERGY, true, PACK>(P, K, R, (unsigned int)I.x_begin,
                                        (unsigned int)(I.x_begin + x_cnt), slot, sh, q, dst, L,
                                        elj, ec);
        if constexpr (PACK) {
            up2(L.fx, L.f0.x, L.f1.x);
            up2(L.fy, L.f0.y, L.f1.y);
            up2(L.fz, L.f0.z, L.f1.z);
        }
        T3<T> fi0 = L.f0, fi1 = L.f1;
        // i forces: sum over the eight slots, then 24 lanes write (atom, component)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            fi0.x += __shfl_xor_sync(FULL, fi0.x, o);
            fi0.y += __shfl_xor_sync(FULL, fi0.y, o);
            fi0.z += __shfl_xor_sync(FULL, fi0.z, o);
            fi1.x += __shfl_xor_sync(FULL, fi1.x, o);
            fi1.y += __shfl_xor_sync(FULL, fi1.y, o);
            fi1.z += __shfl_xor_sync(FULL, fi1.z, o);
        }
        if (slot < 6) {
            const T3<T> f = slot < 3 ? fi0 : fi1;
            const int cpt = slot % 3;
            const T v = cpt == 0 ? f.x : (cpt == 1 ? f.y : f.z);
            if (v != (T)0) {
                long long* d = cpt == 0 ? P.fx : (cpt == 1 ? P.fy : P.fz);
                const int a = I.c * CL + q + (slot < 3 ? 0 : 4);
                add_fixed(d + a, (sizeof(T) == 4) ? to_fixed((float)v) : to_fixed_d((double)v));
            }
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
        const Atom<T> ai0 = load_atom<T>(P, a0, R, K);
        const Atom<T> ai1 = load_atom<T>(P, a0 + 4, R, K);
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
            Atom<T> aj = load_atom<T>(P, ja, R, K);
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
        const Atom<T> ai[2] = {load_atom<T>(P, a0, R, K),
                               load_atom<T>(P, a0 + 4, R, K)};
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
            Atom<T> aj = load_atom<T>(P, ja, R, K);
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
// Environment pairs through the inner rows (the list the force kernel walks),
// in the force kernel's lane layout; the item's computed pairs (64 per round
// of 8 rows, in units of 32) go to pair_cnt[2 R] for the lane efficiency.
__global__ void __launch_bounds__(128) k_count_rows(DevPtrs P) {
    const int lane = threadIdx.x & 31, q = lane & 3, slot = lane >> 2;
    const int n_items = min(*(volatile int*)&P.cnt->n_ritems, P.cap_ritems);
    const int stride = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += stride) {
        const RowItem I = P.ritems[it];
        const int rep = P.rep_of_cl[I.c];
        const RepDev& R = P.reps[rep];
        int cnt = 0;
        long long lanes = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const unsigned int b = pass ? (unsigned int)I.x_begin : I.r_begin;
            const int n = pass ? (I.cnt >> 16) : (I.cnt & 0xFFFF);
            lanes += 64LL * ((n + ROWS_PER_ROUND - 1) / ROWS_PER_ROUND);  // 8 rows x 8 i atoms
            for (unsigned int k = b + slot; k < b + (unsigned int)n; k += ROWS_PER_ROUND) {
                unsigned int word, em = 0u;
                if (pass) {
                    const int2 xr = P.xrows[k];
                    word = (unsigned int)xr.x;
                    em = (unsigned int)xr.y;
                } else {
                    word = P.rows[k];
                }
                const int ja = (int)(word & ROW_SLOT_MASK), code = (int)(word >> ROW_SLOT_BITS);
                float4 xj = P.xq[ja];
                xj.x += (float)(code % 3 - 1) * R.box[0];
                xj.y += (float)((code / 3) % 3 - 1) * R.box[1];
                xj.z += (float)(code / 9 - 1) * R.box[2];
                const bool jreal = P.orig[ja] >= 0;
                for (int h = 0; h < 2; ++h) {
                    const int ii = q + 4 * h;
                    const int a = I.c * CL + ii;
                    const float4 xi = P.xq[a];
                    const float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (!((em >> ii) & 1u) && r2 < P.rc2 && jreal && P.orig[a] >= 0) {
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
    const int n_items = min(*(volatile int*)&P.cnt->n_items_lig, P.cap_items_lig);
    const int stride = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += stride) {
        const Item I = P.items_lig[it];
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
                       int block, int packed) {
    if (precision == 1) {
        k_env_rows<double, true, false><<<grid, block, 0, s>>>(P);
        return;
    }
    if (energy) k_env_rows<float, true, false><<<grid, block, 0, s>>>(P);
    else if (packed) k_env_rows<float, false, true><<<grid, block, 0, s>>>(P);
    else k_env_rows<float, false, false><<<grid, block, 0, s>>>(P);
}

int env_kernel_occupancy(int group, int block, int precision, bool energy, int packed) {
    (void)group;
    int nb = 0;
    if (precision == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<double, true, false>, block, 0);
    else if (energy)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<float, true, false>, block, 0);
    else if (packed)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<float, false, true>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_env_rows<float, false, false>, block, 0);
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
    k_count_rows<<<grid, block, 0, s>>>(P);
    k_count_lig<<<grid, block, 0, s>>>(P);
}

}  // namespace abfe
