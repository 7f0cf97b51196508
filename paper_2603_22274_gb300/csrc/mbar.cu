// MBAR free energies of the states of one window segment (Shirts & Chodera
// 2008), the estimator the paper applies within each GPU segment before summing
// the segments ("Simulation protocol").
//
// The dimensionless free energies solve
//     f_i = -ln sum_n exp(-u_in) / sum_k N_k exp(f_k - u_kn),   f_0 = 0,
// for the K x N matrix of reduced potentials u_kn, by self-consistent
// iteration in FP64 with every iteration on the device. One iteration applies
// the map above once, in one of two exact arrangements:
//  A (log space): ld_n = ln sum_k exp(ln N_k + f_k - u_kn) per sample, then per
//    state f_i = -ln sum_n exp(-u_in - ld_n); 2 K N exponentials.
//  B (scaled linear): with a reference f^r and the stored matrix
//    c_kn = exp(f^r_k - u_kn - b_n), b_n = max over sampled k of f^r_k - u_kn,
//    D_n = sum_k N_k exp(f_k - f^r_k) c_kn and f_i = f^r_i - ln sum_n c_in / D_n;
//    two FP64 matrix-vector passes, no exponential per element.
// B is the same map (multiply numerator and denominator by exp(-b_n)); c_kn
// lies in [0, 1] with a 1 for the largest sampled term of every sample, so D_n
// cannot underflow while |f - f^r| stays moderate. The first iteration is A;
// then c is refreshed from the current f (K N exponentials once) and B runs,
// going back to A and a refresh whenever f drifts more than 20 from f^r or a
// sum is not finite. The state machine lives in device memory: every kernel of
// the loop body checks the mode and returns at once when it is not its turn,
// and the body is a CUDA graph while-node, so there are no host round trips.
// The log-sum-exps take the maximum first and skip terms more than 60 below it
// (relative weight < 1e-26). Reductions have a fixed order: deterministic.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "abfe.h"
#include "abfe_internal.cuh"

namespace {

constexpr int MB_THREADS = 256;
constexpr int MB_CHUNK = 16384;        // samples per partial of k_mbar_part
constexpr double MB_SKIP = -60.0;      // exp(x - max) not evaluated below this

enum : int { MODE_A = 0, MODE_REFRESH = 1, MODE_B = 2 };
constexpr double MB_DRIFT = 20.0;      // refresh c when max |f - f^r| exceeds this

struct MbarDev {
    const double* u;       // [K][N]
    double* c;             // [K][N] scaled weights of arrangement B
    long long N;
    int K, nch;
    const double* logN;    // [K] ln N_k (-inf for N_k = 0)
    double* lognf;         // [K] ln N_k + f_k
    double* f;             // [K]
    double* fr;            // [K] reference f of c
    double* ld;            // [N] ld_n (A) or 1 / D_n (B)
    double2* part;         // [K][nch] (max, sum) (A) or (sum, -) (B)
    int* iter;             // iterations done
    int* status;           // bit 0 converged, bit 1 non-finite
    int* mode;             // MODE_*
    double tol;
    int max_iter;
};

__device__ __forceinline__ double block_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = sh[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, sh[i]);
    return t;  // all threads
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    return t;  // all threads
}

// ld_n for every sample (thread per sample; u rows read coalesced)
__global__ void __launch_bounds__(MB_THREADS) k_mbar_ld(MbarDev M) {
    if (*M.mode != MODE_A) return;
    extern __shared__ double s_lognf[];
    for (int k = threadIdx.x; k < M.K; k += blockDim.x) s_lognf[k] = M.lognf[k];
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < M.N; n += stride) {
        double m = -INFINITY;
        for (int k = 0; k < M.K; ++k) {
            const double a = s_lognf[k];
            if (a > -INFINITY) m = fmax(m, a - M.u[(long long)k * M.N + n]);
        }
        double s = 0.0;
        for (int k = 0; k < M.K; ++k) {
            const double a = s_lognf[k];
            if (a > -INFINITY) {
                const double x = a - M.u[(long long)k * M.N + n] - m;
                if (x > MB_SKIP) s += exp(x);
            }
        }
        const double v = m + log(s);
        M.ld[n] = v;
        if (!isfinite(v)) atomicOr(M.status, 2);
    }
}

// partial log-sum-exp of -u_in - ld_n over one chunk of samples, per state i
__global__ void __launch_bounds__(MB_THREADS) k_mbar_part(MbarDev M) {
    if (*M.mode != MODE_A) return;
    __shared__ double sh[MB_THREADS / 32];
    const int i = blockIdx.y, j = blockIdx.x;
    const long long n0 = (long long)j * MB_CHUNK;
    const long long n1 = n0 + MB_CHUNK < M.N ? n0 + MB_CHUNK : M.N;
    const double* ui = M.u + (long long)i * M.N;
    double m = -INFINITY;
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) m = fmax(m, -ui[n] - M.ld[n]);
    m = block_max(m, sh);
    double s = 0.0;
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) {
        const double x = -ui[n] - M.ld[n] - m;
        if (x > MB_SKIP) s += exp(x);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) M.part[(long long)i * M.nch + j] = make_double2(m, s);
}

// c_kn = exp(f_k - u_kn - b_n) at the current f, which becomes the reference
__global__ void __launch_bounds__(MB_THREADS) k_mbar_refresh(MbarDev M) {
    if (*M.mode != MODE_REFRESH) return;
    extern __shared__ double s_f[];   // [K] f, [K] 1 if sampled
    for (int k = threadIdx.x; k < M.K; k += blockDim.x) {
        s_f[k] = M.f[k];
        s_f[M.K + k] = M.logN[k] > -INFINITY ? 1.0 : 0.0;
    }
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < M.N; n += stride) {
        double b = -INFINITY;
        for (int k = 0; k < M.K; ++k)
            if (s_f[M.K + k] != 0.0) b = fmax(b, s_f[k] - M.u[(long long)k * M.N + n]);
        for (int k = 0; k < M.K; ++k) {
            const double x = s_f[k] - M.u[(long long)k * M.N + n] - b;
            M.c[(long long)k * M.N + n] = x > -745.0 ? exp(x) : 0.0;
        }
    }
}

// after the refresh kernel: f^r = f, switch to B (one thread, stream order)
__global__ void k_mbar_refresh_done(MbarDev M) {
    if (*M.mode != MODE_REFRESH) return;
    for (int k = threadIdx.x; k < M.K; k += blockDim.x) M.fr[k] = M.f[k];
    __syncthreads();
    if (threadIdx.x == 0) *M.mode = MODE_B;
}

// 1 / D_n, D_n = sum_k N_k exp(f_k - f^r_k) c_kn
__global__ void __launch_bounds__(MB_THREADS) k_mbar_gemv_d(MbarDev M) {
    if (*M.mode != MODE_B) return;
    extern __shared__ double s_w[];
    for (int k = threadIdx.x; k < M.K; k += blockDim.x)
        s_w[k] = M.logN[k] > -INFINITY ? exp(M.logN[k] + M.f[k] - M.fr[k]) : 0.0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < M.N; n += stride) {
        double d = 0.0;
        for (int k = 0; k < M.K; ++k) d = fma(s_w[k], M.c[(long long)k * M.N + n], d);
        M.ld[n] = 1.0 / d;
    }
}

// partial sum_n c_in / D_n over one chunk of samples, per state i
__global__ void __launch_bounds__(MB_THREADS) k_mbar_gemv_s(MbarDev M) {
    if (*M.mode != MODE_B) return;
    __shared__ double sh[MB_THREADS / 32];
    const int i = blockIdx.y, j = blockIdx.x;
    const long long n0 = (long long)j * MB_CHUNK;
    const long long n1 = n0 + MB_CHUNK < M.N ? n0 + MB_CHUNK : M.N;
    const double* ci = M.c + (long long)i * M.N;
    double s = 0.0;
    for (long long n = n0 + threadIdx.x; n < n1; n += blockDim.x) s = fma(ci[n], M.ld[n], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) M.part[(long long)i * M.nch + j] = make_double2(s, 0.0);
}

// combine the partials, normalise, test convergence, choose the next mode and
// set the loop condition
__global__ void k_mbar_update(MbarDev M, cudaGraphConditionalHandle h, int use_handle) {
    extern __shared__ double s_fn[];
    __shared__ double sh[32];
    const int mode = *M.mode;
    for (int i = threadIdx.x; i < M.K; i += blockDim.x) {
        const double2* p = M.part + (long long)i * M.nch;
        if (mode == MODE_A) {
            double mx = -INFINITY;
            for (int j = 0; j < M.nch; ++j) mx = fmax(mx, p[j].x);
            double s = 0.0;
            for (int j = 0; j < M.nch; ++j) s += p[j].y * exp(p[j].x - mx);
            s_fn[i] = -(mx + log(s));
        } else {
            double s = 0.0;
            for (int j = 0; j < M.nch; ++j) s += p[j].x;
            s_fn[i] = M.fr[i] - log(s);
        }
    }
    __syncthreads();
    const double f0 = s_fn[0];
    double d = 0.0, drift = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < M.K; i += blockDim.x) {
        const double fi = s_fn[i] - f0;
        if (!isfinite(fi)) bad = true;
        d = fmax(d, fabs(fi - M.f[i]));
        if (mode == MODE_B) drift = fmax(drift, fabs(fi - M.fr[i]));
    }
    const int bad_any = __syncthreads_or(bad);
    if (bad_any && mode == MODE_B) {
        // a sum left the range of arrangement B: redo this iteration in log space
        if (threadIdx.x == 0) {
            *M.mode = MODE_A;
            if (use_handle) cudaGraphSetConditional(h, 1u);
        }
        return;
    }
    for (int i = threadIdx.x; i < M.K; i += blockDim.x) {
        const double fi = s_fn[i] - f0;
        M.f[i] = fi;
        M.lognf[i] = M.logN[i] > -INFINITY ? M.logN[i] + fi : -INFINITY;
    }
    d = block_max(bad_any ? INFINITY : d, sh);
    drift = block_max(drift, sh);
    if (threadIdx.x == 0) {
        const int it = *M.iter + 1;
        *M.iter = it;
        int st = *M.status;
        if (bad_any) st |= 2;
        if (d < M.tol) st |= 1;
        *M.status = st;
        if (mode == MODE_A || drift > MB_DRIFT) *M.mode = MODE_REFRESH;
        const bool go = !(st & 3) && it < M.max_iter;
        if (use_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
    }
}

// non-finite inputs would otherwise drop out of the max-first sums unnoticed
__global__ void k_mbar_check(MbarDev M) {
    const long long total = (long long)M.K * M.N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    bool bad = false;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride)
        bad |= !isfinite(M.u[t]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(M.status, 2);
}

__global__ void k_mbar_init(MbarDev M) {
    for (int i = threadIdx.x; i < M.K; i += blockDim.x) {
        M.f[i] = 0.0;
        M.lognf[i] = M.logN[i];
    }
    if (threadIdx.x == 0) {
        *M.iter = 0;
        *M.status = 0;
        *M.mode = MODE_A;
    }
}

struct Scratch {
    std::vector<std::pair<void*, size_t>> a;
    cudaStream_t s;
    bool ok = true;
    template <class T>
    T* get(size_t n) {
        const size_t b = n * sizeof(T);
        void* p = abfe::lib_alloc(b, s);
        if (!p) ok = false;
        a.push_back({p, b});
        return (T*)p;
    }
    ~Scratch() {
        cudaStreamSynchronize(s);
        for (auto& x : a) abfe::lib_free(x.first, x.second, s);
    }
};

cudaStream_t mbar_stream() {
    // one stream for every call, so that allocator pools tied to a stream are reused
    static std::once_flag once;
    static cudaStream_t s = nullptr;
    std::call_once(once, [] {
        if (cudaStreamCreate(&s) != cudaSuccess) {
            cudaGetLastError();
            s = nullptr;
        }
    });
    return s;
}

abfe_status fail(abfe_status st, const std::string& m) {
    abfe::set_free_error(m.c_str());
    return st;
}

void enqueue_iteration(const MbarDev& M, cudaStream_t s, int grid_ld, cudaGraphConditionalHandle h,
                       int use_handle) {
    k_mbar_refresh<<<grid_ld, MB_THREADS, 2 * sizeof(double) * M.K, s>>>(M);
    k_mbar_refresh_done<<<1, 256, 0, s>>>(M);
    k_mbar_ld<<<grid_ld, MB_THREADS, sizeof(double) * M.K, s>>>(M);
    k_mbar_part<<<dim3(M.nch, M.K), MB_THREADS, 0, s>>>(M);
    k_mbar_gemv_d<<<grid_ld, MB_THREADS, sizeof(double) * M.K, s>>>(M);
    k_mbar_gemv_s<<<dim3(M.nch, M.K), MB_THREADS, 0, s>>>(M);
    k_mbar_update<<<1, 1024, sizeof(double) * M.K, s>>>(M, h, use_handle);
}

abfe_status mbar_run(const double* u_src, bool u_host, const int32_t* N_k, int32_t K, int64_t N,
                     double tol, int32_t max_iter, double* f_out, int32_t* n_iter,
                     cudaStream_t caller) {
    if (!u_src || !N_k || !f_out) return fail(ABFE_ERR_INVALID_ARG, "mbar: NULL pointer");
    if (K < 1 || K > ABFE_MBAR_MAX_K || N < 1 || !(tol > 0.0) || max_iter < 1)
        return fail(ABFE_ERR_INVALID_ARG,
                    "mbar: need 1 <= K <= ABFE_MBAR_MAX_K, N >= 1, tol > 0, max_iter >= 1");
    int64_t tot = 0;
    std::vector<double> logN(K);
    for (int k = 0; k < K; ++k) {
        if (N_k[k] < 0) return fail(ABFE_ERR_INVALID_ARG, "mbar: negative N_k");
        tot += N_k[k];
        logN[k] = N_k[k] > 0 ? std::log((double)N_k[k]) : -INFINITY;
    }
    if (tot != N) return fail(ABFE_ERR_INVALID_ARG, "mbar: sum of N_k differs from N");
    cudaStream_t s = mbar_stream();
    if (!s) return fail(ABFE_ERR_CUDA, "mbar: stream creation failed");
    cudaEvent_t ev = nullptr;
    if (caller) {
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ev, caller) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess) {
            if (ev) cudaEventDestroy(ev);
            cudaGetLastError();
            return fail(ABFE_ERR_CUDA, "mbar: cannot order after the caller's stream");
        }
    }
    MbarDev M{};
    M.N = N;
    M.K = K;
    M.nch = (int)((N + MB_CHUNK - 1) / MB_CHUNK);
    M.tol = tol;
    M.max_iter = max_iter;
    Scratch sc;
    sc.s = s;
    double* d_u = u_host ? sc.get<double>((size_t)K * N) : nullptr;
    double* d_logN = sc.get<double>(K);
    M.lognf = sc.get<double>(K);
    M.f = sc.get<double>(K);
    M.fr = sc.get<double>(K);
    M.c = sc.get<double>((size_t)K * N);
    M.ld = sc.get<double>(N);
    M.part = sc.get<double2>((size_t)K * M.nch);
    int* d_ints = sc.get<int>(3);
    if (ev) cudaEventDestroy(ev);
    if (!sc.ok) return fail(ABFE_ERR_OUT_OF_MEMORY, "mbar: device scratch");
    M.iter = d_ints;
    M.status = d_ints + 1;
    M.mode = d_ints + 2;
    M.logN = d_logN;
    if (u_host) {
        if (cudaMemcpyAsync(d_u, u_src, sizeof(double) * (size_t)K * N, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return fail(ABFE_ERR_CUDA, "mbar: copy of u_kn");
        M.u = d_u;
    } else {
        M.u = u_src;
    }
    if (cudaMemcpyAsync(d_logN, logN.data(), sizeof(double) * K, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return fail(ABFE_ERR_CUDA, "mbar: copy of ln N_k");
    k_mbar_init<<<1, 1024, 0, s>>>(M);
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (N + MB_THREADS - 1) / MB_THREADS;
    const int grid_ld = (int)(want < (long long)n_sm * 8 ? want : (long long)n_sm * 8);
    k_mbar_check<<<n_sm * 4, MB_THREADS, 0, s>>>(M);
    {
        int h_st = 0;
        if (cudaMemcpyAsync(&h_st, M.status, sizeof h_st, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return fail(ABFE_ERR_CUDA, "mbar: input check");
        if (h_st & 2) return fail(ABFE_ERR_NONFINITE, "mbar: non-finite u_kn");
    }

    // the whole iteration as one graph: while (condition) { ld; partials; update }
    bool graph_done = false;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t gx = nullptr;
    if (cudaGraphCreate(&g, 0) == cudaSuccess) {
        cudaGraphConditionalHandle h;
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node;
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            if (cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess) {
                cudaGraph_t body = np.conditional.phGraph_out[0];
                cudaStream_t cs = nullptr;
                if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
                    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed) == cudaSuccess) {
                        enqueue_iteration(M, cs, grid_ld, h, 1);
                        const bool cap = cudaStreamEndCapture(cs, &body) == cudaSuccess;
                        if (cap && cudaGraphInstantiate(&gx, g, 0) == cudaSuccess &&
                            cudaGraphLaunch(gx, s) == cudaSuccess)
                            graph_done = true;
                    }
                    cudaStreamDestroy(cs);
                }
            }
        }
    }
    if (!graph_done) {
        cudaGetLastError();
        // host-driven fallback: the update kernel still tests convergence on the
        // device; the host looks at the flags every 16 iterations
        int h_ints[2] = {0, 0};
        for (int it = 0; it < max_iter;) {
            const int batch = std::min(16, max_iter - it);
            for (int b = 0; b < batch; ++b) enqueue_iteration(M, s, grid_ld, 0, 0);
            it += batch;
            if (cudaMemcpyAsync(h_ints, d_ints, sizeof h_ints, cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                break;
            if (h_ints[1] & 3) break;
        }
    }
    int h_ints[2] = {0, 0};
    cudaMemcpyAsync(h_ints, d_ints, sizeof h_ints, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(f_out, M.f, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(ABFE_ERR_CUDA, std::string("mbar: ") + cudaGetErrorString(e));
    if (n_iter) *n_iter = h_ints[0];
    if (h_ints[1] & 2) return fail(ABFE_ERR_NONFINITE, "mbar: non-finite u_kn or free energy");
    return ABFE_OK;
}

}  // namespace

extern "C" {

abfe_status abfe_mbar(const double* h_u_kn, const int32_t* h_N_k, int32_t K, int64_t N,
                      double tol, int32_t max_iter, double* h_f_k, int32_t* h_n_iter) {
    return mbar_run(h_u_kn, true, h_N_k, K, N, tol, max_iter, h_f_k, h_n_iter, nullptr);
}

abfe_status abfe_mbar_device(const double* d_u_kn, const int32_t* h_N_k, int32_t K, int64_t N,
                             double tol, int32_t max_iter, double* h_f_k, int32_t* h_n_iter,
                             void* stream) {
    return mbar_run(d_u_kn, false, h_N_k, K, N, tol, max_iter, h_f_k, h_n_iter,
                    (cudaStream_t)stream);
}

}  // extern "C"
