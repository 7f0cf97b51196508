// Smooth particle-mesh Ewald (Essmann et al. 1995): the reciprocal-space part
// of the paper's PME electrostatics ("Additional methodological details"), with
// the self energy and the excluded-pair correction, for every window at once.
//
// Per window r a K1 x K2 x K3 grid (K = 2^a 3^b 5^c, at most PME_KMAX), stored
// x fastest: index i1 + K1 (i2 + K2 i3). Charges are q sqrt(k_e), so energies
// come out in kJ/mol.
//   k_pme_spread   (per atom)   cardinal B-splines of order p at the scaled
//                               fractional coordinates u = K x / L; Q += q W1 W2 W3
//                               as 64-bit fixed point (integer atomics: the grid is
//                               independent of the order of the additions)
//   k_pme_fft      (per tile)   3D FFT as three passes of 1D FFTs; a tile is 16
//                               neighbouring lines so that its loads and stores
//                               cover whole 128-byte segments, each warp runs two
//                               lines' mixed-radix (4, 2, 3, 5) Stockham FFTs in
//                               shared memory; the inverse is conj(FFT(conj(.)))
//                               without the 1/N. The forward transform's first
//                               pass reads the fixed-point grid itself (converted
//                               to FP32, then cleared for the next spreading)
//   k_pme_conv     (per point)  E = 1/2 sum_m B(m) C(m) |F(Q)(m)|^2 in FP64 (energy
//                               steps), and F(Q) *= B C in FP32 for the potential
//   k_pme_gather   (per atom)   F_j = -q_j sum_k phi(k) grad(W1 W2 W3), plus the
//                               force of the excluded-pair correction
//                               -k_e q_i q_j erf(beta r)/r from each of the atom's
//                               excluded partners (no atomics on the partner)
//   k_pme_excl     (per atom)   the same correction's energy split by pair kind
// with C(m) = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2) (C(0) = 0) and
// B(m) = |b1(m1)|^2 |b2(m2)|^2 |b3(m3)|^2 from the host's moduli tables.
#include <cuda_runtime.h>

#include <cstdint>

#include "abfe_internal.cuh"

namespace abfe {

namespace {

constexpr double PME_QINV = 1.0 / 1099511627776.0;   // charge grid: 2^40 fixed point
constexpr int FFT_LINES = PME_FFT_LINES;         // lines per FFT block
constexpr int FFT_WARPS = 8;                     // warps per FFT block (FFT_LINES / 2 lines each)
static_assert(FFT_LINES == 16, "k_pme_fft splits element indexes as e & 15, e >> 4");

__device__ __forceinline__ int charge_is_ligand(const DevPtrs& P, const RepDev& R, int o) {
    return P.sys_lig[R.sys_atom_off + o];
}

// charge (times sqrt(k_e)) of an atom in a spreading mode:
// 0 own state (ligand x lambda_q), 1 environment only, 2 ligand only, 3 all at 1
__device__ __forceinline__ float mode_charge(float q, bool lig, float lam_q, int mode) {
    switch (mode) {
        case 0: return lig ? q * lam_q : q;
        case 1: return lig ? 0.f : q;
        case 2: return lig ? q : 0.f;
        default: return q;
    }
}

// B-spline weights W[t] = M_p(w + t) and derivatives D[t] = M_p'(w + t) for
// t = 0..p-1, w in [0, 1) (Cox-de Boor: M_n(x) = (x M_{n-1}(x) + (n-x) M_{n-1}(x-1))/(n-1))
template <int PO>
__device__ __forceinline__ void bspline_wd(float w, float (&W)[PO], float (&D)[PO]) {
    float a[PO];
    a[0] = 1.f;
#pragma unroll
    for (int t = 1; t < PO; ++t) a[t] = 0.f;
#pragma unroll
    for (int n = 2; n <= PO; ++n) {
        if (n == PO) {
            // derivative from order PO-1: M_p'(x) = M_{p-1}(x) - M_{p-1}(x-1)
#pragma unroll
            for (int t = 0; t < PO; ++t) D[t] = (t < PO - 1 ? a[t] : 0.f) - (t > 0 ? a[t - 1] : 0.f);
        }
        const float inv = 1.f / (float)(n - 1);
#pragma unroll
        for (int t = PO - 1; t >= 0; --t) {
            if (t < n) {
                const float x = w + (float)t;
                const float hi = (t < n - 1) ? a[t] : 0.f;
                const float lo = (t > 0) ? a[t - 1] : 0.f;
                a[t] = (x * hi + ((float)n - x) * lo) * inv;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < PO; ++t) W[t] = a[t];
}

__device__ __forceinline__ void frac_coord(float x, float L, int K, int& base, float& w) {
    float u = x / L;
    u -= floorf(u);
    u *= (float)K;
    // a non-finite coordinate (reported by the step's finiteness check) must
    // still index inside the grid
    if (!(u >= 0.f && u < (float)K)) u = (u == (float)K) ? 0.f : (u >= 0.f ? u : 0.f);
    if (!(u < (float)K)) u = 0.f;
    base = (int)floorf(u);
    if (base >= K) base -= K;
    if (base < 0) base = 0;
    w = u - floorf(u);
}

// round to nearest (ties to even) float -> int64 from 32-bit conversions only:
// |x| = h 2^32 + r with h = trunc(|x| 2^-32) and r = |x| - h 2^32 exact in FP32
// (r < 2^32 is a multiple of the ulp of |x|), then r rounded; the same value as
// a direct 64-bit conversion, whose instruction is the slow one
__device__ __forceinline__ long long f2ll_rn_split(float x) {
    const float ax = fabsf(x);
    const float h = truncf(ax * 2.3283064365386963e-10f);   // 2^-32
    const float r = fmaf(-h, 4294967296.0f, ax);
    const unsigned long long v =
        ((unsigned long long)(unsigned)h << 32) + (unsigned long long)__float2uint_rn(r);
    return x < 0.f ? -(long long)v : (long long)v;
}

template <int PO>
__global__ void __launch_bounds__(256) k_pme_spread(DevPtrs P, PmeDev M, int mode) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        const int o = P.orig[s];
        if (o < 0) continue;
        const int r = P.rep_of_cl[s >> 3];
        const RepDev& R = P.reps[r];
        const float4 x = P.xq[s];
        const float q = mode_charge(x.w, charge_is_ligand(P, R, o) != 0, R.lam_q, mode);
        if (q == 0.f) continue;
        const int4 K = M.dims[r];
        int b0, b1, b2;
        float w0, w1, w2;
        frac_coord(x.x, R.box[0], K.x, b0, w0);
        frac_coord(x.y, R.box[1], K.y, b1, w1);
        frac_coord(x.z, R.box[2], K.z, b2, w2);
        float W0[PO], W1[PO], W2[PO], D[PO];
        bspline_wd<PO>(w0, W0, D);
        bspline_wd<PO>(w1, W1, D);
        bspline_wd<PO>(w2, W2, D);
        long long* g = M.qgrid + M.goff[r];
#pragma unroll
        for (int t2 = 0; t2 < PO; ++t2) {
            int k2 = b2 - t2;
            if (k2 < 0) k2 += K.z;
#pragma unroll
            for (int t1 = 0; t1 < PO; ++t1) {
                int k1 = b1 - t1;
                if (k1 < 0) k1 += K.y;
                const float q12 = q * W2[t2] * W1[t1];
                const long long row = (long long)K.x * (k1 + (long long)K.y * k2);
#pragma unroll
                for (int t0 = 0; t0 < PO; ++t0) {
                    int k0 = b0 - t0;
                    if (k0 < 0) k0 += K.x;
                    // FP32 product, scaled by the exact 2^40: no FP64 arithmetic per contribution
                    const long long v = f2ll_rn_split(q12 * W0[t0] * 1099511627776.0f);
                    atomicAdd(reinterpret_cast<unsigned long long*>(g + row + k0),
                              static_cast<unsigned long long>(v));
                }
            }
        }
    }
}

// FP64 copy for the energy split: comp 0 -> real part, comp 1 -> imaginary part
__global__ void k_pme_load_d(PmeDev M, int comp) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < M.total; i += stride) {
        const long long v = M.qgrid[i];
        M.qgrid[i] = 0;
        const double f = (double)v * PME_QINV;
        if (comp == 0) M.dgrid[i] = make_double2(f, 0.0);
        else M.dgrid[i].y = f;
    }
}

// fixed-point grid value v (2^40 units) as float, from the two 32-bit halves
// (32-bit conversions only; the high half, |hi| < 2^24 for any grid value
// within range, converts exactly)
__device__ __forceinline__ float fixed_to_float(long long v) {
    const float hi = (float)(int)(v >> 32);
    const float lo = (float)(unsigned)(v & 0xffffffffll);
    return fmaf(hi, 0.00390625f, lo * 9.094947017729282e-13f);   // 2^-8, 2^-40
}

// complex helpers for float2 (force path) and double2 (energy split)
template <class C> struct cx;
template <> struct cx<float2> {
    using R = float;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ void sc(float x, float* s, float* c) { sincospif(x, s, c); }
};
template <> struct cx<double2> {
    using R = double;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ void sc(double x, double* s, double* c) { sincospi(x, s, c); }
};

template <class C>
__device__ __forceinline__ C cmul(C a, C b) {
    return cx<C>::mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// one Stockham stage of radix RAD on a line of n points (warp-cooperative)
// tw[k] = exp(-2 pi i k / n), k < n, in shared memory
// small integers: q = floor(j / d) from a float reciprocal (exact for j < 2^20)
__device__ __forceinline__ int fdiv(int j, float inv_d) { return (int)(((float)j + 0.5f) * inv_d); }

// y_s = sum_r v_r exp(-2 pi i r s / RAD), s = 0..RAD-1
template <int RAD, class C>
__device__ __forceinline__ void butterfly(const C (&v)[RAD], C (&y)[RAD]) {
    using T = typename cx<C>::R;
    if (RAD == 2) {
        y[0] = cx<C>::mk(v[0].x + v[1].x, v[0].y + v[1].y);
        y[1] = cx<C>::mk(v[0].x - v[1].x, v[0].y - v[1].y);
    } else if (RAD == 4) {
        const C a = cx<C>::mk(v[0].x + v[2].x, v[0].y + v[2].y);
        const C b = cx<C>::mk(v[0].x - v[2].x, v[0].y - v[2].y);
        const C c = cx<C>::mk(v[1].x + v[3].x, v[1].y + v[3].y);
        const C d = cx<C>::mk(v[1].x - v[3].x, v[1].y - v[3].y);   // times -i below
        y[0] = cx<C>::mk(a.x + c.x, a.y + c.y);
        y[2] = cx<C>::mk(a.x - c.x, a.y - c.y);
        y[1] = cx<C>::mk(b.x + d.y, b.y - d.x);
        y[3] = cx<C>::mk(b.x - d.y, b.y + d.x);
    } else if (RAD == 3) {
        // y1,2 = v0 - (v1 + v2)/2 -+ i (sqrt3/2)(v1 - v2)
        const T h = (T)0.8660254037844386;
        const C t1 = cx<C>::mk(v[1].x + v[2].x, v[1].y + v[2].y);
        const C t2 = cx<C>::mk(v[0].x - (T)0.5 * t1.x, v[0].y - (T)0.5 * t1.y);
        const C d = cx<C>::mk(h * (v[1].x - v[2].x), h * (v[1].y - v[2].y));
        y[0] = cx<C>::mk(v[0].x + t1.x, v[0].y + t1.y);
        y[1] = cx<C>::mk(t2.x + d.y, t2.y - d.x);
        y[2] = cx<C>::mk(t2.x - d.y, t2.y + d.x);
    } else {
        // radix 5 with c_k = cos(2 pi k/5), s_k = sin(2 pi k/5):
        // y1,4 = v0 + c1 t1 + c2 t2 -+ i (s1 t3 + s2 t4), y2,3 = v0 + c2 t1 + c1 t2 -+ i (s2 t3 - s1 t4)
        const T c1 = (T)0.30901699437494745, c2 = (T)-0.8090169943749475;
        const T s1 = (T)0.9510565162951535, s2 = (T)0.5877852522924731;
        const C t1 = cx<C>::mk(v[1].x + v[4].x, v[1].y + v[4].y);
        const C t2 = cx<C>::mk(v[2].x + v[3].x, v[2].y + v[3].y);
        const C t3 = cx<C>::mk(v[1].x - v[4].x, v[1].y - v[4].y);
        const C t4 = cx<C>::mk(v[2].x - v[3].x, v[2].y - v[3].y);
        y[0] = cx<C>::mk(v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y);
        const C a1 = cx<C>::mk(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        const C a2 = cx<C>::mk(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        const C b1 = cx<C>::mk(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y);
        const C b2 = cx<C>::mk(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y);
        y[1] = cx<C>::mk(a1.x + b1.y, a1.y - b1.x);
        y[4] = cx<C>::mk(a1.x - b1.y, a1.y + b1.x);
        y[2] = cx<C>::mk(a2.x + b2.y, a2.y - b2.x);
        y[3] = cx<C>::mk(a2.x - b2.y, a2.y + b2.x);
    }
}

// One radix-RAD Stockham stage of NL lines at once (line q at src/dst + q lstr;
// the lines' loads are issued together and share the twiddles).
template <int RAD, int NL, class C>
__device__ __forceinline__ void fft_stage(const C* src, C* dst, int lstr, const C* tw, int n, int Ns, int lane) {
    const int m = n / RAD;
    const int step = n / (Ns * RAD);   // twiddle exponent jm r / (Ns RAD) of a turn = (jm r step) / n
    const float inv_ns = 1.0f / (float)Ns;
    for (int j = lane; j < m; j += 32) {
        const int jq = fdiv(j, inv_ns);
        const int jm = j - jq * Ns;
        C v[NL][RAD], wr[RAD];
#pragma unroll
        for (int q = 0; q < NL; ++q)
#pragma unroll
            for (int r = 0; r < RAD; ++r) v[q][r] = src[q * lstr + j + r * m];
#pragma unroll
        for (int r = 1; r < RAD; ++r) wr[r] = tw[jm * r * step];
        const int idxD = jq * Ns * RAD + jm;
#pragma unroll
        for (int q = 0; q < NL; ++q) {
#pragma unroll
            for (int r = 1; r < RAD; ++r) v[q][r] = cmul(v[q][r], wr[r]);
            C y[RAD];
            butterfly<RAD>(v[q], y);
#pragma unroll
            for (int r = 0; r < RAD; ++r) dst[q * lstr + idxD + r * Ns] = y[r];
        }
    }
}

__device__ __forceinline__ int fft_radix(int rem) {
    if (rem % 4 == 0) return 4;
    if (rem % 2 == 0) return 2;
    if (rem % 3 == 0) return 3;
    return 5;
}

// number of stages of an n-point transform: its parity says which buffer holds the result
__device__ __forceinline__ int fft_stages(int n) {
    int c = 0;
    for (int rem = n; rem > 1; rem /= fft_radix(rem)) ++c;
    return c;
}

template <int NL, class C>
__device__ void fft_line(C* b0, C* b1, int lstr, const C* tw, int n, int lane) {
    C* src = b0;
    C* dst = b1;
    int Ns = 1, rem = n;
    while (rem > 1) {
        const int R = fft_radix(rem);
        switch (R) {
            case 4: fft_stage<4, NL>(src, dst, lstr, tw, n, Ns, lane); break;
            case 2: fft_stage<2, NL>(src, dst, lstr, tw, n, Ns, lane); break;
            case 3: fft_stage<3, NL>(src, dst, lstr, tw, n, Ns, lane); break;
            default: fft_stage<5, NL>(src, dst, lstr, tw, n, Ns, lane); break;
        }
        __syncwarp();
        C* t = src;
        src = dst;
        dst = t;
        Ns *= R;
        rem /= R;
    }
}

template <class C> __device__ __forceinline__ const C* tw_table(const PmeDev& M);
template <> __device__ __forceinline__ const float2* tw_table<float2>(const PmeDev& M) { return M.twf; }
template <> __device__ __forceinline__ const double2* tw_table<double2>(const PmeDev& M) { return M.twd; }

// shared memory of one FFT block: two buffers of FFT_LINES lines, each line
// padded to an odd stride (n + 1) so that the 16 lines' elements k fall in
// different banks, and the twiddle table
__host__ __device__ constexpr int fft_smem_elems(int kmax) { return 2 * FFT_LINES * (kmax + 1) + kmax; }

// FIXED: the pass reads the fixed-point charge grid (real input), clears it
// for the next spreading, and writes its result to `grid`
template <class C, bool FIXED>
__global__ void __launch_bounds__(FFT_WARPS * 32) k_pme_fft(PmeDev M, C* grid, int axis, int inverse) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    C* s_fft = reinterpret_cast<C*>(s_raw);
    const int g = blockIdx.x;
    const int r = M.tile_rep[axis][g];
    const int4 K = M.dims[r];
    // line axis (n points, stride stn), the axis the lines of a tile run along
    // (b, stride stb), and the remaining one (c, stride stc)
    const int n = axis == 0 ? K.x : (axis == 1 ? K.y : K.z);
    const int nb = axis == 0 ? K.y : K.x;
    const int stn = axis == 0 ? 1 : (axis == 1 ? K.x : K.x * K.y);
    const int stb = axis == 0 ? K.x : 1;
    const int stc = axis == 2 ? K.x : K.x * K.y;
    const int nbt = (nb + FFT_LINES - 1) / FFT_LINES;
    const int lt = g - M.tiles[axis][r];
    const int tb = lt % nbt, tc = lt / nbt;
    C* gbase = grid + M.goff[r] + (long long)tc * stc;
    const int ls = n + 1;
    C* buf0 = s_fft;
    C* buf1 = s_fft + FFT_LINES * ls;
    C* s_tw = s_fft + 2 * FFT_LINES * ls;
    const C* twg = tw_table<C>(M) + M.tw_off[n];
    for (int k = threadIdx.x; k < n; k += blockDim.x) s_tw[k] = twg[k];
    const int total = FFT_LINES * n;
    const float inv_n = 1.0f / (float)n;
    // element e -> line t, point k (lines of axis 0 are contiguous rows: k runs
    // fastest; otherwise the 16 lines are neighbours in memory: t runs fastest)
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int t, k;
        if (axis == 0) { t = fdiv(e, inv_n); k = e - t * n; } else { t = e & (FFT_LINES - 1); k = e >> 4; }
        const int b = tb * FFT_LINES + t;
        if (b < nb) {
            C v;
            if (FIXED) {
                const long long q = M.qgrid[(gbase - grid) + k * stn + b * stb];
                v = cx<C>::mk((typename cx<C>::R)fixed_to_float(q), 0);
            } else {
                v = gbase[k * stn + b * stb];
                if (inverse) v.y = -v.y;
            }
            buf0[t * ls + k] = v;
        }
    }
    if (FIXED) {
        // cleared after all of this thread's loads, so that they stay independent
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            int t, k;
            if (axis == 0) { t = fdiv(e, inv_n); k = e - t * n; } else { t = e & (FFT_LINES - 1); k = e >> 4; }
            const int b = tb * FFT_LINES + t;
            if (b < nb) M.qgrid[(gbase - grid) + k * stn + b * stb] = 0;
        }
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int l = w; l < FFT_LINES; l += FFT_WARPS)
        if (tb * FFT_LINES + l < nb) fft_line<1>(buf0 + l * ls, buf1 + l * ls, 0, s_tw, n, lane);
    __syncthreads();
    // all lines of a tile have the same length: the stage count's parity picks the buffer
    const C* res = (fft_stages(n) & 1) ? buf1 : buf0;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int t, k;
        if (axis == 0) { t = fdiv(e, inv_n); k = e - t * n; } else { t = e & (FFT_LINES - 1); k = e >> 4; }
        const int b = tb * FFT_LINES + t;
        if (b < nb) {
            C v = res[t * ls + k];
            if (inverse) v.y = -v.y;
            gbase[k * stn + b * stb] = v;
        }
    }
}

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;   // thread 0
}

// CONV_CPB 256-point chunks per block (M.chunks: prefix per replica; a block's
// chunks may belong to different replicas). Forces need only F(Q) *= B C,
// done in FP32; the energy, on energy steps, is summed in FP64 per chunk.
constexpr int CONV_CPB = 4;
__global__ void __launch_bounds__(256) k_pme_conv(DevPtrs P, PmeDev M, int ea_slot, int multiply) {
    __shared__ double sh[8];
    const int g0 = blockIdx.x * CONV_CPB;
    double bc[CONV_CPB];
    float2 F[CONV_CPB];
    long long gi[CONV_CPB];
    int rr[CONV_CPB];
#pragma unroll
    for (int c = 0; c < CONV_CPB; ++c) {
        const int g = g0 + c;
        gi[c] = -1;
        rr[c] = 0;
        bc[c] = 0.0;
        F[c] = make_float2(0.f, 0.f);
        if (g < M.n_chunks) {
            const int r = M.chunk_rep[g];
            rr[c] = r;
            const int n_pts = (int)(M.goff[r + 1] - M.goff[r]);
            const int i = (g - M.chunks[r]) * 256 + threadIdx.x;
            if (i < n_pts) {
                gi[c] = M.goff[r] + i;
                bc[c] = M.infl[M.infl_off[P.reps[r].sys] + i];   // B(m) C(m)
                F[c] = M.cgrid[gi[c]];
            }
        }
    }
    if (multiply) {
#pragma unroll
        for (int c = 0; c < CONV_CPB; ++c) {
            if (gi[c] >= 0) {
                const float b = (float)bc[c];
                M.cgrid[gi[c]] = make_float2(F[c].x * b, F[c].y * b);
            }
        }
    }
    if (ea_slot >= 0) {
#pragma unroll
        for (int c = 0; c < CONV_CPB; ++c) {
            if (g0 + c >= M.n_chunks) break;   // uniform over the block
            const double e = gi[c] >= 0 ? 0.5 * bc[c] * ((double)F[c].x * F[c].x + (double)F[c].y * F[c].y) : 0.0;
            const double t = block_sum_d(e, sh);
            if (threadIdx.x == 0) add_fixed(P.eacc + (size_t)rr[c] * EA_N + ea_slot, to_fixed_d(t));
        }
    }
}

// Split of the reciprocal energy by charge kind from one transform of
// z = Q_env + i Q_lig (both real): F_env(m) = (F_z(m) + conj F_z(-m)) / 2 and
// F_lig(m) = (F_z(m) - conj F_z(-m)) / 2i. With E(lambda) = 1/2 sum B C
// |F_env + lambda F_lig|^2 = A + lambda B + lambda^2 C:
// A = 1/2 sum BC |F_env|^2, B = sum BC Re(F_env conj F_lig), C = 1/2 sum BC |F_lig|^2.
// B comes from the cross term directly, not as a difference of large totals.
__global__ void __launch_bounds__(256) k_pme_conv_split(DevPtrs P, PmeDev M) {
    __shared__ double sh[8];
    const int g = blockIdx.x;
    const int r = M.chunk_rep[g];
    const int n_pts = (int)(M.goff[r + 1] - M.goff[r]);
    const int i = (g - M.chunks[r]) * 256 + threadIdx.x;
    const RepDev& R = P.reps[r];
    const int4 K = M.dims[r];
    double ea = 0.0, eb = 0.0, ec = 0.0;
    if (i < n_pts) {
        const int i1 = i % K.x;
        const int i2 = (i / K.x) % K.y;
        const int i3 = i / (K.x * K.y);
        const double bc = M.infl[M.infl_off[R.sys] + i];
        if (bc != 0.0) {
            const int j1 = i1 ? K.x - i1 : 0, j2 = i2 ? K.y - i2 : 0, j3 = i3 ? K.z - i3 : 0;
            const double2 z = M.dgrid[M.goff[r] + i];
            const double2 zm = M.dgrid[M.goff[r] + j1 + K.x * (j2 + K.y * j3)];
            // F_env = (z + conj zm) / 2, F_lig = (z - conj zm) / (2 i)
            const double er = 0.5 * (z.x + zm.x), ei = 0.5 * (z.y - zm.y);
            const double lr = 0.5 * (z.y + zm.y), li = -0.5 * (z.x - zm.x);
            ea = 0.5 * bc * (er * er + ei * ei);
            eb = bc * (er * lr + ei * li);
            ec = 0.5 * bc * (lr * lr + li * li);
        }
    }
    const double ta = block_sum_d(ea, sh);
    const double tb = block_sum_d(eb, sh);
    const double tc = block_sum_d(ec, sh);
    if (threadIdx.x == 0) {
        long long* a = P.eacc + (size_t)r * EA_N;
        add_fixed(a + EA_REC_ENV, to_fixed_d(ta));
        add_fixed(a + EA_REC_MIX, to_fixed_d(tb));
        add_fixed(a + EA_REC_LIG, to_fixed_d(tc));
    }
}

template <int PO>
__global__ void __launch_bounds__(256) k_pme_gather(DevPtrs P, PmeDev M, int energy) {
    const int stride = gridDim.x * blockDim.x;
    const float beta = (float)M.beta;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        const int o = P.orig[s];
        if (o < 0) continue;
        const int r = P.rep_of_cl[s >> 3];
        const RepDev& R = P.reps[r];
        const float4 x = P.xq[s];
        const float q = mode_charge(x.w, charge_is_ligand(P, R, o) != 0, R.lam_q, 0);
        if (q == 0.f) continue;
        const int4 K = M.dims[r];
        int b0, b1, b2;
        float w0, w1, w2;
        frac_coord(x.x, R.box[0], K.x, b0, w0);
        frac_coord(x.y, R.box[1], K.y, b1, w1);
        frac_coord(x.z, R.box[2], K.z, b2, w2);
        float W0[PO], W1[PO], W2[PO], D0[PO], D1[PO], D2[PO];
        bspline_wd<PO>(w0, W0, D0);
        bspline_wd<PO>(w1, W1, D1);
        bspline_wd<PO>(w2, W2, D2);
        const float2* g = M.cgrid + M.goff[r];
        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
        for (int t2 = 0; t2 < PO; ++t2) {
            int k2 = b2 - t2;
            if (k2 < 0) k2 += K.z;
#pragma unroll
            for (int t1 = 0; t1 < PO; ++t1) {
                int k1 = b1 - t1;
                if (k1 < 0) k1 += K.y;
                const long long row = (long long)K.x * (k1 + (long long)K.y * k2);
                float sx = 0.f, sw = 0.f;
#pragma unroll
                for (int t0 = 0; t0 < PO; ++t0) {
                    int k0 = b0 - t0;
                    if (k0 < 0) k0 += K.x;
                    const float phi = g[row + k0].x;
                    sx = fmaf(phi, D0[t0], sx);
                    sw = fmaf(phi, W0[t0], sw);
                }
                gx = fmaf(sx, W1[t1] * W2[t2], gx);
                gy = fmaf(sw, D1[t1] * W2[t2], gy);
                gz = fmaf(sw, W1[t1] * D2[t2], gz);
            }
        }
        float fx = -q * gx * (float)K.x / R.box[0];
        float fy = -q * gy * (float)K.y / R.box[1];
        float fz = -q * gz * (float)K.z / R.box[2];
        // excluded-pair correction E = -qq erf(beta r)/r, r = |x_j - x_i|; the
        // force on this atom is dE/dr (x_j - x_i)/r. Every excluded pair is in
        // both atoms' lists; its energy is counted by the lower index.
        const int kb = P.sys_ex_off[R.sys_ex_off + o], ke = P.sys_ex_off[R.sys_ex_off + o + 1];
        double e_ex = 0.0;
        for (int kk = kb; kk < ke; ++kk) {
            const int j = P.sys_ex_idx[kk];
            if (j == o) continue;
            const float4 xj = P.xq[P.slot_of[R.atom_off + j]];
            const float qq = q * mode_charge(xj.w, charge_is_ligand(P, R, j) != 0, R.lam_q, 0);
            if (qq == 0.f) continue;
            float dx = xj.x - x.x, dy = xj.y - x.y, dz = xj.z - x.z;
            dx -= R.box[0] * rintf(dx / R.box[0]);
            dy -= R.box[1] * rintf(dy / R.box[1]);
            dz -= R.box[2] * rintf(dz / R.box[2]);
            const float r2 = dx * dx + dy * dy + dz * dz;
            const float rr = sqrtf(r2);
            const float dEdr = -qq * (1.1283791670955126f * beta * expf(-beta * beta * r2) / rr - erff(beta * rr) / r2);
            const float fs = dEdr / rr;
            fx = fmaf(fs, dx, fx);
            fy = fmaf(fs, dy, fy);
            fz = fmaf(fs, dz, fz);
            if (energy && j > o) {
                const double ddx = dx, ddy = dy, ddz = dz;
                const double rd = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
                e_ex -= (double)qq * erf(M.beta * rd) / rd;
            }
        }
        if (e_ex != 0.0) add_fixed(P.eacc + (size_t)r * EA_N + EA_EXCL, to_fixed_d(e_ex));
        add_fixed(P.fx + s, to_fixed(fx));
        add_fixed(P.fy + s, to_fixed(fy));
        add_fixed(P.fz + s, to_fixed(fz));
    }
}

// Excluded-pair correction energies with unit ligand charges, split by pair
// kind into EA_EXCL_ENV (env-env), EA_EXCL_MIX (env-ligand, scales as
// lambda_q) and EA_EXCL_LIG (ligand-ligand, lambda_q^2).
__global__ void __launch_bounds__(256) k_pme_excl(DevPtrs P, PmeDev M) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.S; s += stride) {
        const int o = P.orig[s];
        if (o < 0) continue;
        const int r = P.rep_of_cl[s >> 3];
        const RepDev& R = P.reps[r];
        const int kb = P.sys_ex_off[R.sys_ex_off + o], ke = P.sys_ex_off[R.sys_ex_off + o + 1];
        if (kb == ke) continue;
        const float4 xi = P.xq[s];
        const bool li = charge_is_ligand(P, R, o) != 0;
        double e_env = 0.0, e_mix = 0.0, e_lig = 0.0;
        for (int kk = kb; kk < ke; ++kk) {
            const int j = P.sys_ex_idx[kk];
            if (j <= o) continue;                       // each pair once, by the lower index
            const float4 xj = P.xq[P.slot_of[R.atom_off + j]];
            const bool lj = charge_is_ligand(P, R, j) != 0;
            float dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
            dx -= R.box[0] * rintf(dx / R.box[0]);
            dy -= R.box[1] * rintf(dy / R.box[1]);
            dz -= R.box[2] * rintf(dz / R.box[2]);
            const double ddx = dx, ddy = dy, ddz = dz;
            const double rd = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
            const double e = -(double)xi.w * (double)xj.w * erf(M.beta * rd) / rd;
            if (li && lj) e_lig += e;
            else if (li || lj) e_mix += e;
            else e_env += e;
        }
        long long* a = P.eacc + (size_t)r * EA_N;
        if (e_env != 0.0) add_fixed(a + EA_EXCL_ENV, to_fixed_d(e_env));
        if (e_mix != 0.0) add_fixed(a + EA_EXCL_MIX, to_fixed_d(e_mix));
        if (e_lig != 0.0) add_fixed(a + EA_EXCL_LIG, to_fixed_d(e_lig));
    }
}

template <int PO>
void spread_gather(const DevPtrs& P, const PmeDev& M, cudaStream_t s, int n_sm, int mode,
                   bool gather, int energy) {
    const int grid = n_sm * 8;
    if (gather) k_pme_gather<PO><<<grid, 256, 0, s>>>(P, M, energy);
    else k_pme_spread<PO><<<grid, 256, 0, s>>>(P, M, mode);
}

void spread_or_gather(const DevPtrs& P, const PmeDev& M, cudaStream_t s, int n_sm, int mode,
                      bool gather, int energy = 0) {
    switch (M.order) {
        case 4: spread_gather<4>(P, M, s, n_sm, mode, gather, energy); break;
        case 5: spread_gather<5>(P, M, s, n_sm, mode, gather, energy); break;
        default: spread_gather<6>(P, M, s, n_sm, mode, gather, energy); break;
    }
}

// from_fixed: the first pass takes its input from the fixed-point charge grid
template <class C>
void fft3d(const PmeDev& M, C* grid, cudaStream_t s, int inverse, bool from_fixed = false) {
    const int smem = (int)(fft_smem_elems(M.kmax) * sizeof(C));
    for (int a = 0; a < 3; ++a) {
        if (M.n_tiles[a] == 0) continue;
        if (a == 0 && from_fixed)
            k_pme_fft<C, true><<<M.n_tiles[a], FFT_WARPS * 32, smem, s>>>(M, grid, a, inverse);
        else
            k_pme_fft<C, false><<<M.n_tiles[a], FFT_WARPS * 32, smem, s>>>(M, grid, a, inverse);
    }
}

// The attribute is a property of the kernel, shared by every context of the
// process: it is set to what the longest possible line needs (a context with
// smaller grids must not lower it under another context's launches); each
// launch asks only for what its own grids need.
template <class C, bool FIXED>
cudaError_t fft_prepare() {
    return cudaFuncSetAttribute(k_pme_fft<C, FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(fft_smem_elems(PME_KMAX) * sizeof(C)));
}

}  // namespace

cudaError_t pme_prepare(PmeDev& M) {
    if (M.kmax > PME_KMAX) return cudaErrorInvalidValue;
    cudaError_t e = fft_prepare<float2, false>();
    if (e == cudaSuccess) e = fft_prepare<float2, true>();
    if (e == cudaSuccess) e = fft_prepare<double2, false>();
    return e;
}

// Reciprocal forces at every replica's own lambda_q (plus the reciprocal and
// excluded-pair energies when `energy`).
void launch_pme_forces(const DevPtrs& P, const PmeDev& M, cudaStream_t s, int n_sm, bool energy) {
    spread_or_gather(P, M, s, n_sm, 0, false);
    fft3d(M, M.cgrid, s, 0, true);
    k_pme_conv<<<(M.n_chunks + CONV_CPB - 1) / CONV_CPB, 256, 0, s>>>(P, M, energy ? EA_REC : -1, 1);
    fft3d(M, M.cgrid, s, 1);
    spread_or_gather(P, M, s, n_sm, 0, true, energy ? 1 : 0);
}

// Energies that make the reciprocal part of u_kn a polynomial in lambda_q,
// E_rec(lambda) = A + lambda B + lambda^2 C: environment charges in the real
// and ligand charges in the imaginary part of one grid, one transform, the
// split in k_pme_conv_split, all in FP64 (an FP32 transform's error scales with
// the environment's much larger amplitudes and would swamp the ligand terms);
// and the excluded-pair terms by pair kind.
void launch_pme_decomposition(const DevPtrs& P, const PmeDev& M, cudaStream_t s, int n_sm) {
    spread_or_gather(P, M, s, n_sm, 1, false);
    k_pme_load_d<<<n_sm * 8, 256, 0, s>>>(M, 0);
    spread_or_gather(P, M, s, n_sm, 2, false);
    k_pme_load_d<<<n_sm * 8, 256, 0, s>>>(M, 1);
    fft3d(M, M.dgrid, s, 0);
    k_pme_conv_split<<<M.n_chunks, 256, 0, s>>>(P, M);
    k_pme_excl<<<n_sm * 8, 256, 0, s>>>(P, M);
}

}  // namespace abfe
