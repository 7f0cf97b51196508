// abfe_ukn_frame_noalloc: the lambda-dependent part of one frame's u_kn row for
// callers that cannot allocate device memory (for example a plugin inside a
// host MD engine whose device memory belongs to the host application's own
// allocator). It uses no context and calls no cudaMalloc/cudaFree: its only
// scratch is the file-scope array below, shared by every call on a device.
//
// Pass 1 (grid n_lig x nbx blocks): each block takes one ligand atom and a
// strided share of all atoms. Per chunk of NA_CH states it walks its atoms
// once: the separation, the cutoff and exclusion tests and (first chunk) the
// unit-charge Coulomb sums are evaluated once per pair, the softcore LJ at
// every lambda_v,k of the chunk accumulates in registers; a fixed-order block
// reduction writes one partial per block and state into the scratch array. A
// ligand index outside [0, n) is never dereferenced: its block writes NaN
// partials, so every du[k] of that call is NaN. Pass 2 (one block): sums the
// partials in block order (deterministic), adds the charge-scaled Coulomb terms
// and lambda_r,k times the Boresch restraint energy, and writes du[k]. All
// arithmetic is FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "abfe.h"

namespace {

constexpr int NA_MAX_BLOCKS = ABFE_NOALLOC_MAX_BLOCKS;
constexpr int NA_MAX_K = ABFE_NOALLOC_MAX_K;
constexpr int NA_SLOTS = NA_MAX_K + 2;  // K LJ sums + ligand-env and ligand-ligand Coulomb
constexpr int NA_THREADS = 128;

// Scratch: one row of NA_SLOTS partial sums per block (about 1 MB). Every
// call overwrites the rows it uses before reading them.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS * NA_SLOTS];

struct NaParams {
    int n, n_lig, K, nbx, mode, has_boresch;
    double box[3], rc2, beta, ke, alpha, p;
    const float* pos;
    const float* q;
    const float* sig;
    const float* eps;
    const unsigned char* lig;
    const int* lig_idx;
    const int* lig_excl;
    double lam_r[NA_MAX_K], lam_q[NA_MAX_K], lam_v[NA_MAX_K], A[NA_MAX_K];
    int anc[6];
    double b_r0, th0[2], ph0[3], kr, kth, kph;
};

__device__ __forceinline__ double mi1(double d, double L) { return d - L * rint(d / L); }

__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;  // valid in thread 0
}

constexpr int NA_CH = 16;  // states per pass over the atoms (register accumulators)

__global__ void __launch_bounds__(NA_THREADS) k_na_pairs(const NaParams P, double* scratch) {
    __shared__ double sh[NA_THREADS / 32];
    __shared__ int excl[ABFE_NOALLOC_MAX_EXCL];
    const int la = blockIdx.y;
    const int a = P.lig_idx[la];
    const int row = blockIdx.y * P.nbx + blockIdx.x;
    if (a < 0 || a >= P.n) {
        // bad ligand index from the caller: flag the whole call through NaN partials
        for (int k = threadIdx.x; k < P.K + 2; k += blockDim.x)
            scratch[(size_t)row * NA_SLOTS + k] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    if (threadIdx.x < ABFE_NOALLOC_MAX_EXCL)
        excl[threadIdx.x] = P.lig_excl[la * ABFE_NOALLOC_MAX_EXCL + threadIdx.x];
    __syncthreads();
    const double xa = P.pos[3 * a], ya = P.pos[3 * a + 1], za = P.pos[3 * a + 2];
    const double qa = P.q[a], sa = P.sig[a], ea = P.eps[a];
    const int stride = P.nbx * blockDim.x;
    const int first = blockIdx.x * blockDim.x + threadIdx.x;
    for (int k0 = 0; k0 < P.K; k0 += NA_CH) {
        const bool coul = k0 == 0;   // the Coulomb sums ride on the first chunk
        double acc[NA_CH];
#pragma unroll
        for (int q = 0; q < NA_CH; ++q) acc[q] = 0.0;
        double cle = 0.0, cll = 0.0;  // ligand-environment, ligand-ligand (unit scale)
        for (int b = first; b < P.n; b += stride) {
            if (b == a) continue;
            const bool bl = P.lig[b] != 0;
            if (bl && b < a) continue;           // each ligand-ligand pair once
            // decoupled ligand-ligand pairs are lambda independent: not part of du
            if (bl && P.mode == 1) continue;
            bool ex = false;
            for (int e = 0; e < ABFE_NOALLOC_MAX_EXCL; ++e) ex |= (excl[e] == b);
            if (ex) continue;
            const double dx = mi1((double)P.pos[3 * b] - xa, P.box[0]);
            const double dy = mi1((double)P.pos[3 * b + 1] - ya, P.box[1]);
            const double dz = mi1((double)P.pos[3 * b + 2] - za, P.box[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < P.rc2)) continue;
            if (coul) {
                const double r = sqrt(r2);
                const double u = P.ke * qa * (double)P.q[b] * erfc(P.beta * r) / r;
                if (bl) cll += u; else cle += u;
            }
            const double s = 0.5 * (sa + (double)P.sig[b]);
            const double s2 = s * s, s6 = s2 * s2 * s2;
            const double e4 = 4.0 * sqrt(ea * (double)P.eps[b]);
            const double r6 = r2 * r2 * r2;
#pragma unroll
            for (int q = 0; q < NA_CH; ++q) {
                if (k0 + q < P.K) {
                    const double x = s6 / (P.A[k0 + q] * s6 + r6);
                    acc[q] += P.lam_v[k0 + q] * e4 * (x * x - x);
                }
            }
        }
        for (int q = 0; q < NA_CH && k0 + q < P.K; ++q) {
            const double t = block_sum(acc[q], sh);
            if (threadIdx.x == 0) scratch[(size_t)row * NA_SLOTS + k0 + q] = t;
        }
        if (coul) {
            const double t1 = block_sum(cle, sh);
            if (threadIdx.x == 0) scratch[(size_t)row * NA_SLOTS + P.K] = t1;
            const double t2 = block_sum(cll, sh);
            if (threadIdx.x == 0) scratch[(size_t)row * NA_SLOTS + P.K + 1] = t2;
        }
    }
}

struct V3 {
    double x, y, z;
};
__device__ V3 vsub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ double vdot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ V3 vcross(V3 a, V3 b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// restraint energy U_B of the six anchors (P1 P2 P3 L1 L2 L3), nearest images
__device__ double boresch_energy(const NaParams& P) {
    V3 p[6];
    for (int i = 0; i < 6; ++i) {
        const int a = P.anc[i];
        p[i] = V3{(double)P.pos[3 * a], (double)P.pos[3 * a + 1], (double)P.pos[3 * a + 2]};
    }
    auto sep = [&](int from, int to) {
        V3 d = vsub(p[to], p[from]);
        d.x = mi1(d.x, P.box[0]); d.y = mi1(d.y, P.box[1]); d.z = mi1(d.z, P.box[2]);
        return d;
    };
    double U = 0.0;
    const V3 d = sep(0, 3);
    const double r = sqrt(vdot(d, d));
    U += 0.5 * P.kr * (r - P.b_r0) * (r - P.b_r0);
    const int ang[2][3] = {{0, 3, 4}, {3, 0, 1}};
    for (int t = 0; t < 2; ++t) {
        const V3 u = sep(ang[t][1], ang[t][0]), v = sep(ang[t][1], ang[t][2]);
        double c = vdot(u, v) / sqrt(vdot(u, u) * vdot(v, v));
        c = fmin(1.0, fmax(-1.0, c));
        const double th = acos(c);
        U += 0.5 * P.kth * (th - P.th0[t]) * (th - P.th0[t]);
    }
    const int dih[3][4] = {{1, 0, 3, 4}, {0, 3, 4, 5}, {3, 0, 1, 2}};
    for (int t = 0; t < 3; ++t) {
        const V3 b1 = sep(dih[t][0], dih[t][1]), b2 = sep(dih[t][1], dih[t][2]),
                 b3 = sep(dih[t][2], dih[t][3]);
        const V3 n1 = vcross(b1, b2), n2 = vcross(b2, b3);
        const double phi = atan2(sqrt(vdot(b2, b2)) * vdot(b1, n2), vdot(n1, n2));
        U += P.kph * (1.0 - cos(phi - P.ph0[t]));
    }
    return U;
}

__global__ void __launch_bounds__(NA_THREADS) k_na_finish(const NaParams P, const double* scratch,
                                                          double* du) {
    __shared__ double s_ub;
    if (threadIdx.x == 0) s_ub = P.has_boresch ? boresch_energy(P) : 0.0;
    __syncthreads();
    const int rows = P.n_lig * P.nbx;
    double cle = 0.0, cll = 0.0;
    for (int r = 0; r < rows; ++r) {
        cle += scratch[(size_t)r * NA_SLOTS + P.K];
        cll += scratch[(size_t)r * NA_SLOTS + P.K + 1];
    }
    for (int k = threadIdx.x; k < P.K; k += blockDim.x) {
        double lj = 0.0;
        for (int r = 0; r < rows; ++r) lj += scratch[(size_t)r * NA_SLOTS + k];
        const double lq = P.lam_q[k];
        du[k] = lj + lq * cle + lq * lq * cll + P.lam_r[k] * s_ub;
    }
}

std::mutex g_na_mutex;
double* g_na_ptr[64] = {nullptr};

}  // namespace

extern "C" abfe_status abfe_ukn_frame_noalloc(const abfe_noalloc_frame* f, double* d_du,
                                              void* cuda_stream) {
    if (!f || !d_du || !f->pos || !f->charge || !f->sigma || !f->epsilon || !f->is_ligand ||
        !f->lig_idx || !f->lig_excl)
        return ABFE_ERR_INVALID_ARG;
    if (f->n_atoms < 1 || f->n_atoms > ABFE_NOALLOC_MAX_ATOMS || f->n_lig < 1 ||
        f->n_lig > ABFE_NOALLOC_MAX_LIG || f->K < 1 || f->K > NA_MAX_K)
        return ABFE_ERR_INVALID_ARG;  // sizes beyond the documented maxima
    if (!(f->cutoff > 0) || !(f->sc_p >= 1.0) || (f->ligand_mode != 0 && f->ligand_mode != 1))
        return ABFE_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(f->cutoff < 0.5 * f->box[d])) return ABFE_ERR_CUTOFF_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return ABFE_ERR_CUDA;
    }
    double* scratch = nullptr;
    {
        // first call on a device: look up the device address of the scratch
        // array with that device current
        std::lock_guard<std::mutex> lk(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return ABFE_ERR_CUDA;
            }
            g_na_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_na_ptr[dev];
    }
    NaParams P;
    P.n = f->n_atoms;
    P.n_lig = f->n_lig;
    P.K = f->K;
    P.nbx = NA_MAX_BLOCKS / f->n_lig;
    if (P.nbx > 4) P.nbx = 4;
    P.mode = f->ligand_mode;
    P.has_boresch = f->has_boresch ? 1 : 0;
    for (int d = 0; d < 3; ++d) P.box[d] = f->box[d];
    P.rc2 = f->cutoff * f->cutoff;
    P.beta = f->ewald_beta;
    P.ke = f->coulomb_k;
    P.alpha = f->sc_alpha;
    P.p = f->sc_p;
    P.pos = f->pos;
    P.q = f->charge;
    P.sig = f->sigma;
    P.eps = f->epsilon;
    P.lig = f->is_ligand;
    P.lig_idx = f->lig_idx;
    P.lig_excl = f->lig_excl;
    for (int k = 0; k < f->K; ++k) {
        const double lr = f->lam_r[k], lq = f->lam_q[k], lv = f->lam_v[k];
        if (!(lr >= 0 && lr <= 1 && lq >= 0 && lq <= 1 && lv >= 0 && lv <= 1))
            return ABFE_ERR_INVALID_ARG;
        P.lam_r[k] = lr;
        P.lam_q[k] = lq;
        P.lam_v[k] = lv;
        P.A[k] = f->sc_alpha * std::pow(1.0 - lv, f->sc_p);
    }
    for (int i = 0; i < 6; ++i) {
        P.anc[i] = f->anchors[i];
        if (P.has_boresch && (P.anc[i] < 0 || P.anc[i] >= P.n)) return ABFE_ERR_INVALID_ARG;
    }
    P.b_r0 = f->b_r0;
    P.th0[0] = f->b_theta0[0]; P.th0[1] = f->b_theta0[1];
    P.ph0[0] = f->b_phi0[0]; P.ph0[1] = f->b_phi0[1]; P.ph0[2] = f->b_phi0[2];
    P.kr = f->b_kr; P.kth = f->b_ktheta; P.kph = f->b_kphi;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_na_pairs<<<dim3(P.nbx, P.n_lig), NA_THREADS, 0, s>>>(P, scratch);
    k_na_finish<<<1, NA_THREADS, 0, s>>>(P, scratch, d_du);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ABFE_OK : ABFE_ERR_CUDA;
}
