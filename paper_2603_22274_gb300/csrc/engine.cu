// Host side of the C ABI (abfe.h): context, device memory, launch sequencing,
// CUDA-graph capture of the step loop, autotuning, checkpoints.
//
// One context holds every replica (lambda window) of every system in one set of
// device arrays; each stage (list build, pair forces, integrator) is a single
// launch over all replicas. The step loop can be captured as a CUDA graph whose
// list rebuild sits in a conditional (IF) node set by the device, so the graph
// runs without host round trips and rebuilds only when an atom moved more than
// half the skin.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "abfe.h"
#include "abfe_internal.cuh"

using namespace abfe;

namespace {

abfe_alloc_fn g_alloc = nullptr;
abfe_free_fn g_free = nullptr;
void* g_user = nullptr;
thread_local std::string g_create_err;

struct SchedHost {
    int K = 0;
    std::vector<double> lr, lq, lv;
    std::vector<int> kvidx;
    std::vector<double> kvals;
};

struct EventPool {
    std::vector<cudaEvent_t> a, b;
    int used = 0;
};

constexpr int SP_PRE = 0, SP_STEP = 1, SP_POST = 2, SP_ZERO = 3, SP_XPOST = 4, SP_XPRE = 5,
              SP_N = 6;
constexpr double PRUNE_SKIN_MAX = 0.15;   // nm: largest inner-list buffer (rows are sized for it)

}  // namespace

struct abfe_ctx {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;
    cudaStream_t fork = nullptr;           // ligand / bonded / restraint branch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int device = 0, n_sm = 0;
    abfe_params prm{};
    abfe_tuning tune{};
    double skin_cap = 0.0;
    int R = 0, NS = 0;
    std::vector<int> sys_of_rep, sched_of_rep, state_of_rep;
    std::vector<int> sys_n, sys_nlig, sys_atom_off, sys_ex_row, sys_bond_off, sys_nbonds, sys_bor,
        sys_nexcl, sys_ntri;
    std::vector<std::array<double, 3>> sys_box;
    std::vector<RepDev> reps_h;
    std::vector<int> rep_of_cl_h;
    std::vector<int64_t> rep_atom_off;
    int64_t total_atoms = 0;
    int S = 0, C = 0, NCOL = 0, max_bonds = 0, n_lig_cl = 0, max_lig_cl = 0, max_tors = 0;
    int n_bond_total = 0;
    int max_aw = 0;
    std::vector<int> sys_tors_off, sys_ntors, sys_aw_off, sys_naw;
    DevPtrs P{};
    std::vector<std::pair<void*, size_t>> allocs;
    int64_t device_bytes = 0;
    RepDev* d_reps = nullptr;
    Counters* d_cnt = nullptr;
    StepParams* d_sp = nullptr;
    double* d_energy = nullptr;
    double* d_dudl = nullptr;
    double* d_ukn = nullptr;
    double* d_du = nullptr;
    int ukn_cap = 0;
    double* d_atom3 = nullptr;
    long long* d_paircnt = nullptr;
    int* d_atomcnt = nullptr;
    dbl4* d_sched_state = nullptr;
    int* d_sched_K = nullptr;
    float* d_kv_lam = nullptr;
    float* d_kv_A = nullptr;
    double* d_kv_dlam = nullptr;
    double* d_kv_dA = nullptr;
    double2* d_sched_sc = nullptr;         // per (schedule, state): softcore A and dA/dlambda_v
    bool pme = false;                      // reciprocal-space Ewald on
    PmeDev pm{};
    // replica exchange: groups of replicas sharing (system, schedule)
    int* d_ex = nullptr;                   // grp[R] | goff[R+1] | slot_rep[R] | held[R] | n_acc
    std::vector<int> ex_goff, ex_held;
    bool ex_unique = true;                 // every group holds distinct states
    int ex_every = 0;                      // steps between in-loop exchange attempts (0 = none)
    uint64_t ex_seed = 0;
    unsigned long long dev_step = 0;       // host mirror of the device step counter
    bool reps_dirty = false;               // device replica states newer than reps_h
    SchedHost sched[MAX_SCHED];
    bool states_set = false, f_valid = false, force_rebuild = true, force_prune = false;
    int64_t steps_done = 0;
    long long lane_groups = 0;
    std::string err;
    int env_grid = 0, lig_grid = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_steps = 0;
    bool g_prof = false;
    int g_mode = 0;  // 1 = conditional rebuild node, 2 = predicated rebuild kernels
    int prof_max = 0;
    EventPool ev_env, ev_lig, ev_int, ev_build, ev_prune;
    std::vector<double> rep_rho;            // atom density of each replica's box
    double rows_skin = -1.0;                // prune skin the inner-row buffer is sized for
    unsigned int* d_row_base = nullptr;     // per replica inner-row regions (set by ensure_rows)
    unsigned int* d_row_cap = nullptr;
};

namespace {

int max_K(abfe_ctx* c);
abfe_status ensure_ukn(abfe_ctx* c, int ld);

abfe_status set_error(abfe_ctx* c, abfe_status s, const std::string& m) {
    if (c) c->err = m;
    else g_create_err = m;
    return s;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_error(c, ABFE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void* dev_alloc(abfe_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, (void*)c->stream, g_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->allocs.push_back({p, bytes});
        c->device_bytes += (int64_t)bytes;
        if (cudaMemsetAsync(p, 0, bytes, c->stream) != cudaSuccess) cudaGetLastError();
    }
    return p;
}

template <class T>
T* dalloc(abfe_ctx* c, size_t n, bool& ok) {
    T* p = (T*)dev_alloc(c, n * sizeof(T));
    if (!p) ok = false;
    return p;
}

void dev_free(abfe_ctx* c, void* p) {
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (c->allocs[k].first != p) continue;
        cudaStreamSynchronize(c->stream);
        if (g_free) g_free(p, c->allocs[k].second, (void*)c->stream, g_user);
        else cudaFree(p);
        c->device_bytes -= (int64_t)c->allocs[k].second;
        c->allocs.erase(c->allocs.begin() + (long)k);
        return;
    }
}

// The inner-row buffer, sized for a prune skin: per cluster 8 atoms x
// (2 pi / 3) rho r^3 half-list partners, r = r_c + prune_skin, over 8 pair
// slots per row at a lane efficiency of at least 0.5, with 10% margin (the
// density taken 5% above the box average for dense cores). Grows (never
// shrinks) when a larger prune skin is set; at most 2^32 - 1 rows.
abfe_status ensure_rows(abfe_ctx* c, double prune_skin) {
    const double ps = std::max(prune_skin, 0.06);
    if (c->P.rows && ps <= c->rows_skin) return ABFE_OK;
    const double r = c->prm.cutoff + ps;
    // one region per replica (pruned separately)
    std::vector<unsigned int> base(c->R), cap(c->R);
    int64_t need = 0;
    for (int q = 0; q < c->R; ++q) {
        const double ppa = (2.0 * M_PI / 3.0) * 1.05 * c->rep_rho[q] * r * r * r;
        const int64_t cq = (int64_t)c->reps_h[q].n_cl_cap * (int64_t)std::ceil(1.1 * ppa / 0.5 + 16.0) + 64;
        base[q] = (unsigned int)std::min<int64_t>(need, UINT32_MAX);
        cap[q] = (unsigned int)std::min<int64_t>(cq, UINT32_MAX);
        need += cq;
    }
    if (need > (int64_t)UINT32_MAX)
        return set_error(c, ABFE_ERR_OUT_OF_MEMORY, "inner list exceeds 2^32 rows (smaller prune_skin)");
    if (c->P.rows) dev_free(c, c->P.rows);
    c->P.rows = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * (size_t)std::max<int64_t>(need, 1));
    if (!c->P.rows) {
        c->P.cap_rows = 0;
        c->rows_skin = -1.0;
        return set_error(c, ABFE_ERR_OUT_OF_MEMORY, "inner list rows");
    }
    if (cudaMemcpyAsync(c->d_row_base, base.data(), sizeof(unsigned int) * c->R,
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->d_row_cap, cap.data(), sizeof(unsigned int) * c->R,
                        cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return set_error(c, ABFE_ERR_CUDA, "inner list regions");
    c->P.cap_rows = (unsigned int)need;
    c->rows_skin = ps;
    c->force_rebuild = true;   // every replica's rows go to its new region
    return ABFE_OK;
}

void free_all(abfe_ctx* c) {
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    cudaStreamSynchronize(c->stream);
    for (auto& a : c->allocs) {
        if (g_free) g_free(a.first, a.second, (void*)c->stream, g_user);
        else cudaFree(a.first);
    }
    c->allocs.clear();
    for (EventPool* ep : {&c->ev_env, &c->ev_lig, &c->ev_int, &c->ev_build, &c->ev_prune}) {
        for (auto e : ep->a) cudaEventDestroy(e);
        for (auto e : ep->b) cudaEventDestroy(e);
        ep->a.clear(); ep->b.clear();
    }
}

// A system's bonds in the order the bond kernel takes them: first every bonded
// triangle (a, b, c) found greedily, as the three bonds (a, b), (a, c), (b, c)
// (a water's O-H, O-H and H-H), then the other bonds as given. A thread takes a
// triangle whole, so its three atoms' forces are summed in registers before
// the fixed-point adds. Returns the number of triangles.
int order_bonds(const abfe_system_desc& d, std::vector<int2>& out, std::vector<float2>& outp) {
    const int nb = d.n_bonds;
    std::vector<std::vector<std::pair<int, int>>> adj(d.n_atoms);   // (partner, bond)
    for (int b = 0; b < nb; ++b) {
        const int i = d.bond_idx[2 * b], j = d.bond_idx[2 * b + 1];
        if (i == j) continue;
        adj[i].push_back({j, b});
        adj[j].push_back({i, b});
    }
    auto find = [&](int i, int j) {
        for (const auto& e : adj[i])
            if (e.first == j) return e.second;
        return -1;
    };
    std::vector<char> used(nb, 0);
    auto put = [&](int i, int j, int b) {
        out.push_back(make_int2(i, j));
        outp.push_back(make_float2((float)d.bond_r0[b], (float)d.bond_k[b]));
        used[b] = 1;
    };
    int n_tri = 0;
    for (int a = 0; a < d.n_atoms; ++a) {
        const auto& na = adj[a];
        for (size_t p = 0; p < na.size(); ++p) {
            if (used[na[p].second]) continue;
            for (size_t q = p + 1; q < na.size(); ++q) {
                if (used[na[q].second] || used[na[p].second]) continue;
                const int b = na[p].first, c2 = na[q].first;
                if (b == c2) continue;
                const int bc = find(b, c2);
                if (bc < 0 || used[bc]) continue;
                put(a, b, na[p].second);
                put(a, c2, na[q].second);
                put(b, c2, bc);
                ++n_tri;
            }
        }
    }
    for (int b = 0; b < nb; ++b)
        if (!used[b]) put(d.bond_idx[2 * b], d.bond_idx[2 * b + 1], b);
    return n_tri;
}

int64_t est_entries_per_cluster(double rho, double rl, int n_cl_rep) {
    const double a = std::cbrt(8.0 / rho) * 1.4;
    const double s = 2.0 * a;
    const double vm = s * s * s + 6 * s * s * rl + 3 * M_PI * s * rl * rl + 4.0 / 3.0 * M_PI * rl * rl * rl;
    const double cnt = vm * rho / 8.0;
    double e = 0.6 * cnt + 16;
    e = std::min(e, 27.0 * n_cl_rep + 16);
    return (int64_t)std::ceil(e);
}

void prof_rec(abfe_ctx* c, EventPool& ep, bool begin, cudaStream_t s) {
    if (!c->prof_max || ep.used >= (int)ep.a.size()) return;
    // inside a stream capture the record must become an event-record node of the graph
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    const unsigned int fl = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (begin) cudaEventRecordWithFlags(ep.a[ep.used], s, fl);
    else { cudaEventRecordWithFlags(ep.b[ep.used], s, fl); ep.used++; }
}

DevPtrs with_sp(const abfe_ctx* c, int slot) {
    DevPtrs P = c->P;
    P.sp = c->d_sp + slot;
    return P;
}

// The small ligand, bond and restraint kernels run on a forked stream next to
// the environment pair kernel (parallel branches when captured in a graph);
// all of them add into the same fixed-point force accumulators.
// (fork = false: everything on s, for captures where the fork stream is busy)
void enqueue_forces(abfe_ctx* c, cudaStream_t s, bool energy, bool fork = true) {
    cudaStream_t f = fork ? c->fork : s;
    if (fork) {
        cudaEventRecord(c->ev_fork, s);
        cudaStreamWaitEvent(c->fork, c->ev_fork, 0);
    }
    if (fork) prof_rec(c, c->ev_lig, true, f);
    launch_lig_forces(c->P, f, c->prm.precision, c->lig_grid, 128, energy);
    if (fork) prof_rec(c, c->ev_lig, false, f);
    launch_bonds(c->P, f, c->prm.precision, energy);
    launch_torsions(c->P, f, c->max_tors);
    launch_boresch(c->P, f);
    if (energy) launch_aw_sums(c->P, f, c->max_aw);
    if (c->pme) {
        launch_pme_forces(c->P, c->pm, f, c->n_sm, energy);
        // energy passes also split the reciprocal energy by charge kind (dU/dlambda_q, u_kn)
        if (energy) launch_pme_decomposition(c->P, c->pm, f, c->n_sm);
    }
    if (fork) cudaEventRecord(c->ev_join, c->fork);
    if (fork) prof_rec(c, c->ev_env, true, s);
    launch_env_forces(c->P, s, energy, c->prm.precision, c->env_grid, c->tune.block_threads);
    if (fork) prof_rec(c, c->ev_env, false, s);
    if (fork) cudaStreamWaitEvent(s, c->ev_join, 0);
}

// zero forces, displacement check, rebuild and prune decisions, (predicated)
// outer rebuild and prune
void enqueue_prepare(abfe_ctx* c, cudaStream_t s) {
    launch_integrate(with_sp(c, SP_ZERO), s, c->n_sm);
    launch_step_end(c->P, s, 0, c->force_rebuild ? 1 : 0, c->force_prune ? 1 : 0, 0, 0, 0, 0);
    // host-forced builds and prunes are timed while profiling is on
    const bool tb = c->force_rebuild, tp = c->force_rebuild || c->force_prune;
    if (tb) prof_rec(c, c->ev_build, true, s);
    launch_rebuild(c->P, s, c->n_sm);
    launch_list_build(c->P, s, c->max_lig_cl);
    if (tb) prof_rec(c, c->ev_build, false, s);
    if (tp) prof_rec(c, c->ev_prune, true, s);
    launch_prune(c->P, s, c->n_sm);
    if (tp) prof_rec(c, c->ev_prune, false, s);
    c->force_rebuild = false;
    c->force_prune = false;
}

abfe_status check_device(abfe_ctx* c) {
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    Counters h;
    CK(cudaMemcpy(&h, c->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost));
    if (h.err == 0) return ABFE_OK;
    int zero = 0;
    CK(cudaMemcpy(&c->d_cnt->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
    char buf[320];
    abfe_status st = ABFE_ERR_CUDA;
    const bool list = (h.err & (ERRB_LIST | ERRB_COLUMN | ERRB_CLUSTERS | ERRB_GROUP)) != 0;
    // err_info belongs to the first error raised; with one flag set it is that flag's
    const bool single = (h.err & (h.err - 1)) == 0;
    if (list) {
        c->force_rebuild = true;
        c->f_valid = false;
    }
    if (h.err & ERRB_NONFINITE) {
        // a non-finite state is the usual cause of the other flags (atoms flying apart)
        st = ABFE_ERR_NONFINITE;
        if (single)
            snprintf(buf, sizeof buf, "non-finite force, energy or coordinate (replica %d)",
                     h.err_info[0]);
        else
            snprintf(buf, sizeof buf,
                     "non-finite force, energy or coordinate, with further device errors "
                     "(flags 0x%x; info of the first error: %d %d %d)",
                     h.err, h.err_info[0], h.err_info[1], h.err_info[2]);
    } else if (list) {
        st = ABFE_ERR_LIST_OVERFLOW;
        static const char* const kinds[] = {"?", "entries", "masked entries", "env items",
                                             "ligand items", "prune item", "rows",
                                             "masked rows", "row items"};
        const int kind = h.err_info[1] & 15;
        if (h.err == ERRB_LIST)
            snprintf(buf, sizeof buf,
                     "neighbour-list capacity exceeded: replica %d, cluster %d, %s region needs %d",
                     h.err_info[1] >> 4, h.err_info[0], kinds[kind <= 8 ? kind : 0],
                     h.err_info[2]);
        else
            snprintf(buf, sizeof buf,
                     "neighbour-list capacity exceeded (flags 0x%x; info of the first error: %d %d %d)",
                     h.err, h.err_info[0], h.err_info[1], h.err_info[2]);
    } else {
        snprintf(buf, sizeof buf, "device error flags 0x%x (info %d %d %d)", h.err,
                 h.err_info[0], h.err_info[1], h.err_info[2]);
    }
    return set_error(c, st, buf);
}

abfe_status need_states(abfe_ctx* c) {
    if (!c->states_set)
        return set_error(c, ABFE_ERR_STATE, "lambda schedule / replica states not set");
    return ABFE_OK;
}

// cardinal B-spline M_p(x) (support [0, p]) in FP64, by its recursion
double bspline_host(int p, double x) {
    if (p == 2) return (x >= 0.0 && x <= 2.0) ? 1.0 - std::fabs(x - 1.0) : 0.0;
    return (x * bspline_host(p - 1, x) + (p - x) * bspline_host(p - 1, x - 1.0)) / (p - 1);
}

// grid sizes, B-spline moduli, self energies and device grids of the smooth PME
abfe_status setup_pme(abfe_ctx* c, const abfe_system_desc* systems, int n_systems, DevPtrs& P) {
    const int po = c->prm.pme_order;
    const double beta = c->prm.ewald_beta, ke = c->prm.coulomb_k;
    auto smooth = [](int k) {
        for (int f : {2, 3, 5})
            while (k % f == 0) k /= f;
        return k == 1;
    };
    std::vector<int4> sdims(n_systems);
    std::vector<double> infl;                  // B(m) C(m) per system and grid point
    std::vector<long long> infl_off(n_systems);
    std::vector<double2> selfv(n_systems);
    std::vector<int> tw_off(PME_KMAX + 1, -1);
    std::vector<double2> twd;
    std::vector<float2> twf;
    for (int si = 0; si < n_systems; ++si) {
        const abfe_system_desc& d = systems[si];
        int Kd[3];
        for (int a = 0; a < 3; ++a) {
            int k = std::max(2 * po, (int)std::ceil(d.box[a] / c->prm.pme_spacing - 1e-9));
            while (!smooth(k)) ++k;
            if (k > PME_KMAX)
                return set_error(nullptr, ABFE_ERR_INVALID_ARG,
                                 "PME grid above 256 points per box edge (increase pme_spacing)");
            Kd[a] = k;
            if (tw_off[k] < 0) {
                // twiddle table of an FFT of length k
                tw_off[k] = (int)twd.size();
                for (int j = 0; j < k; ++j) {
                    const double ang = -2.0 * M_PI * j / k;
                    twd.push_back(make_double2(std::cos(ang), std::sin(ang)));
                    twf.push_back(make_float2((float)std::cos(ang), (float)std::sin(ang)));
                }
            }
        }
        sdims[si] = make_int4(Kd[0], Kd[1], Kd[2], 0);
        // B-spline moduli |b_a(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) exp(2 pi i m k / K_a)|^2
        std::vector<double> bm[3];
        for (int a = 0; a < 3; ++a) {
            const int K = Kd[a];
            bm[a].resize(K);
            for (int m = 0; m < K; ++m) {
                double re = 0.0, im = 0.0;
                for (int k = 0; k <= po - 2; ++k) {
                    const double w = bspline_host(po, k + 1.0), ang = 2.0 * M_PI * m * k / K;
                    re += w * std::cos(ang);
                    im += w * std::sin(ang);
                }
                bm[a][m] = 1.0 / (re * re + im * im);
            }
        }
        // influence function C(m) = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), C(0) = 0
        infl_off[si] = (long long)infl.size();
        const double V = d.box[0] * d.box[1] * d.box[2];
        for (int i3 = 0; i3 < Kd[2]; ++i3)
            for (int i2 = 0; i2 < Kd[1]; ++i2)
                for (int i1 = 0; i1 < Kd[0]; ++i1) {
                    const int f1 = i1 <= Kd[0] / 2 ? i1 : i1 - Kd[0];
                    const int f2 = i2 <= Kd[1] / 2 ? i2 : i2 - Kd[1];
                    const int f3 = i3 <= Kd[2] / 2 ? i3 : i3 - Kd[2];
                    const double m1 = f1 / d.box[0], m2 = f2 / d.box[1], m3 = f3 / d.box[2];
                    const double msq = m1 * m1 + m2 * m2 + m3 * m3;
                    double bc = 0.0;
                    if (msq > 0.0)
                        bc = bm[0][i1] * bm[1][i2] * bm[2][i3] *
                             std::exp(-M_PI * M_PI * msq / (beta * beta)) / (M_PI * V * msq);
                    infl.push_back(bc);
                }
        double s_env = 0.0, s_lig = 0.0;
        for (int i = 0; i < d.n_atoms; ++i) {
            const double q2 = d.charge[i] * d.charge[i];
            if (d.is_ligand && d.is_ligand[i]) s_lig += q2; else s_env += q2;
        }
        const double f = -ke * beta / std::sqrt(M_PI);
        selfv[si] = make_double2(f * s_env, f * s_lig);
    }
    const int R = c->R;
    std::vector<int4> dims(R);
    std::vector<long long> goff(R + 1, 0);
    std::vector<int> tiles(3 * (R + 1), 0), chunks(R + 1, 0);
    for (int r = 0; r < R; ++r) {
        const int4 K = sdims[c->reps_h[r].sys];
        dims[r] = K;
        const long long pts = (long long)K.x * K.y * K.z;
        goff[r + 1] = goff[r] + pts;
        chunks[r + 1] = chunks[r] + (int)((pts + 255) / 256);
        const int Ka[3] = {K.x, K.y, K.z};
        for (int a = 0; a < 3; ++a) {
            const int b = a == 0 ? 1 : 0, cc = a == 2 ? 1 : 2;
            tiles[a * (R + 1) + r + 1] =
                tiles[a * (R + 1) + r] + ((Ka[b] + PME_FFT_LINES - 1) / PME_FFT_LINES) * Ka[cc];
        }
    }
    int kmax = 1;
    for (int r = 0; r < R; ++r) kmax = std::max(kmax, std::max(dims[r].x, std::max(dims[r].y, dims[r].z)));
    bool ok = true;
    PmeDev& M = c->pm;
    M.R = R;
    M.order = po;
    M.kmax = kmax;
    if (pme_prepare(M) != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, ABFE_ERR_CUDA, "PME FFT kernel attributes");
    }
    M.total = goff[R];
    M.n_chunks = chunks[R];
    M.beta = beta;
    int4* d_dims = dalloc<int4>(c, R, ok);
    long long* d_goff = dalloc<long long>(c, R + 1, ok);
    int* d_tiles = dalloc<int>(c, 3 * (R + 1), ok);
    int* d_chunks = dalloc<int>(c, R + 1, ok);
    // replica of every FFT tile and convolution chunk (one load instead of a search)
    std::vector<int> tile_rep[3], chunk_rep(chunks[R]);
    for (int a = 0; a < 3; ++a) {
        tile_rep[a].resize(tiles[a * (R + 1) + R]);
        for (int r = 0; r < R; ++r)
            for (int t = tiles[a * (R + 1) + r]; t < tiles[a * (R + 1) + r + 1]; ++t) tile_rep[a][t] = r;
    }
    for (int r = 0; r < R; ++r)
        for (int t = chunks[r]; t < chunks[r + 1]; ++t) chunk_rep[t] = r;
    int* d_tile_rep[3];
    for (int a = 0; a < 3; ++a) d_tile_rep[a] = dalloc<int>(c, tile_rep[a].size(), ok);
    int* d_chunk_rep = dalloc<int>(c, chunk_rep.size(), ok);
    double* d_infl = dalloc<double>(c, infl.size(), ok);
    long long* d_infl_off = dalloc<long long>(c, n_systems, ok);
    double2* d_twd = dalloc<double2>(c, twd.size(), ok);
    float2* d_twf = dalloc<float2>(c, twf.size(), ok);
    int* d_tw_off = dalloc<int>(c, PME_KMAX + 1, ok);
    double2* d_self = dalloc<double2>(c, n_systems, ok);
    M.qgrid = dalloc<long long>(c, M.total, ok);
    M.cgrid = dalloc<float2>(c, M.total, ok);
    M.dgrid = dalloc<double2>(c, M.total, ok);
    if (!ok) return set_error(nullptr, ABFE_ERR_OUT_OF_MEMORY, "PME grids");
    cudaError_t e = cudaSuccess;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
    };
    up(d_dims, dims.data(), sizeof(int4) * R);
    up(d_goff, goff.data(), sizeof(long long) * (R + 1));
    up(d_tiles, tiles.data(), sizeof(int) * tiles.size());
    up(d_chunks, chunks.data(), sizeof(int) * (R + 1));
    for (int a = 0; a < 3; ++a) up(d_tile_rep[a], tile_rep[a].data(), sizeof(int) * tile_rep[a].size());
    up(d_chunk_rep, chunk_rep.data(), sizeof(int) * chunk_rep.size());
    up(d_infl, infl.data(), sizeof(double) * infl.size());
    up(d_infl_off, infl_off.data(), sizeof(long long) * n_systems);
    up(d_twd, twd.data(), sizeof(double2) * twd.size());
    up(d_twf, twf.data(), sizeof(float2) * twf.size());
    up(d_tw_off, tw_off.data(), sizeof(int) * (PME_KMAX + 1));
    up(d_self, selfv.data(), sizeof(double2) * n_systems);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(nullptr, ABFE_ERR_CUDA, std::string("PME upload: ") + cudaGetErrorString(e));
    }
    M.dims = d_dims;
    M.goff = d_goff;
    for (int a = 0; a < 3; ++a) {
        M.tiles[a] = d_tiles + a * (R + 1);
        M.n_tiles[a] = tiles[a * (R + 1) + R];
    }
    M.chunks = d_chunks;
    M.chunk_rep = d_chunk_rep;
    for (int a = 0; a < 3; ++a) M.tile_rep[a] = d_tile_rep[a];
    M.infl = d_infl;
    M.infl_off = d_infl_off;
    M.twd = d_twd;
    M.twf = d_twf;
    M.tw_off = d_tw_off;
    P.pme_self = d_self;
    return ABFE_OK;
}

void update_grids(abfe_ctx* c) {
    c->P.rlist = (float)(c->prm.cutoff + c->tune.skin);
    const double rin = c->prm.cutoff + c->tune.prune_skin + 1e-5;   // slack above FP32 rounding
    c->P.rin2 = (float)(rin * rin);
    c->P.skin_out_half2 = (float)(0.25 * c->tune.skin * c->tune.skin);
    c->P.skin_in_half2 = (float)(0.25 * c->tune.prune_skin * c->tune.prune_skin);
    int occ = env_kernel_occupancy(c->tune.block_threads, c->prm.precision, false);
    if (occ < 1) occ = 1;
    c->env_grid = c->n_sm * occ;
    c->lig_grid = c->n_sm * 4;
    c->P.group = c->prm.precision == 1 ? 1 : c->tune.group;
    c->P.max_entries = c->tune.max_entries;
}

abfe_status upload_reps(abfe_ctx* c) {
    CK(cudaMemcpyAsync(c->d_reps, c->reps_h.data(), sizeof(RepDev) * c->R, cudaMemcpyHostToDevice,
                       c->stream));
    return ABFE_OK;
}

bool finite3(const double* p, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

namespace abfe {

void* lib_alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, (void*)s, g_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

void lib_free(void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (g_free) g_free(p, bytes, (void*)s, g_user);
    else cudaFree(p);
}

void set_free_error(const char* msg) { g_create_err = msg ? msg : ""; }

}  // namespace abfe

// ============================================================================ C ABI

extern "C" {

void abfe_set_allocator(abfe_alloc_fn a, abfe_free_fn f, void* user) {
    g_alloc = a;
    g_free = f;
    g_user = user;
}

const char* abfe_status_string(abfe_status s) {
    switch (s) {
        case ABFE_OK: return "ok";
        case ABFE_ERR_INVALID_ARG: return "invalid argument";
        case ABFE_ERR_CUTOFF_TOO_LARGE: return "cutoff too large for the box";
        case ABFE_ERR_LIST_OVERFLOW: return "neighbour list overflow";
        case ABFE_ERR_NONFINITE: return "non-finite value";
        case ABFE_ERR_CUDA: return "CUDA error";
        case ABFE_ERR_TIMEOUT: return "device wait timed out";
        case ABFE_ERR_NOT_IMPLEMENTED: return "not implemented";
        case ABFE_ERR_STATE: return "call out of order";
        case ABFE_ERR_OUT_OF_MEMORY: return "out of device memory";
    }
    return "unknown status";
}

const char* abfe_last_error(const abfe_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }
int32_t abfe_num_replicas(const abfe_ctx* c) { return c ? c->R : 0; }
int64_t abfe_total_atoms(const abfe_ctx* c) { return c ? c->total_atoms : 0; }
int64_t abfe_atom_offset(const abfe_ctx* c, int32_t r) {
    return (c && r >= 0 && r < c->R) ? c->rep_atom_off[r] : -1;
}

abfe_status abfe_create(const abfe_system_desc* systems, int32_t n_systems,
                        const int32_t* system_of_replica, int32_t n_replicas,
                        const abfe_params* p, void* cuda_stream, abfe_ctx** out) {
    abfe_ctx* c = nullptr;
    g_create_err.clear();
    if (!out) return set_error(nullptr, ABFE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!systems || n_systems < 1 || !system_of_replica || n_replicas < 1 || !p)
        return set_error(nullptr, ABFE_ERR_INVALID_ARG, "NULL or empty systems/replicas/params");
    if (n_replicas > 65535) return set_error(nullptr, ABFE_ERR_INVALID_ARG, "at most 65535 replicas");
    if (!(p->cutoff > 0) || !(p->ewald_beta >= 0) || !(p->sc_alpha >= 0) || !(p->sc_p >= 1.0) ||
        !(p->kT > 0) || !(p->skin >= 0) || !(p->coulomb_k >= 0) ||
        (p->ligand_mode != 0 && p->ligand_mode != 1) || (p->precision != 0 && p->precision != 1))
        return set_error(nullptr, ABFE_ERR_INVALID_ARG,
                         "bad parameters (cutoff>0, beta>=0, alpha>=0, p>=1, kT>0, skin>=0, "
                         "ligand_mode 0/1, precision 0/1)");
    if (!(p->pme_order == 0 || (p->pme_order >= 4 && p->pme_order <= 6)) ||
        (p->pme_order > 0 && !(p->pme_spacing > 0.0 && p->ewald_beta > 0.0)))
        return set_error(nullptr, ABFE_ERR_INVALID_ARG,
                         "pme_order 0 or 4..6 with pme_spacing > 0 and ewald_beta > 0");
    if (p->pme_order > 0 && p->ligand_mode != 0)
        return set_error(nullptr, ABFE_ERR_NOT_IMPLEMENTED,
                         "reciprocal-space Ewald needs ligand_mode 0 (annihilation)");
    if (p->precision == 0 && p->ewald_beta * p->cutoff > ABFE_ERFC_TMAX)
        return set_error(nullptr, ABFE_ERR_INVALID_ARG,
                         "FP32 pair arithmetic needs ewald_beta*cutoff <= 3.6 (use precision=1)");
    for (int r = 0; r < n_replicas; ++r)
        if (system_of_replica[r] < 0 || system_of_replica[r] >= n_systems)
            return set_error(nullptr, ABFE_ERR_INVALID_ARG, "system_of_replica out of range");
    const double rlist = p->cutoff + p->skin;
    // lists are sized for the largest skin the cadence tuner may choose
    double min_edge = 1e30;
    for (int s = 0; s < n_systems; ++s)
        for (int k = 0; k < 3; ++k) min_edge = std::min(min_edge, systems[s].box[k]);
    const double skin_cap = std::max(p->skin, std::min(0.3, 0.98 * min_edge - p->cutoff));
    const double rlist_cap = p->cutoff + skin_cap;
    for (int s = 0; s < n_systems; ++s) {
        const abfe_system_desc& d = systems[s];
        if (d.n_atoms < 1 || !d.pos || !d.mass || !d.charge || !d.sigma || !d.epsilon || !d.is_ligand)
            return set_error(nullptr, ABFE_ERR_INVALID_ARG, "system " + std::to_string(s) + ": NULL array or no atoms");
        for (int k = 0; k < 3; ++k) {
            if (!(d.box[k] > 0)) return set_error(nullptr, ABFE_ERR_INVALID_ARG, "box edge <= 0");
            if (!(p->cutoff < 0.5 * d.box[k]))
                return set_error(nullptr, ABFE_ERR_CUTOFF_TOO_LARGE,
                                 "cutoff must be < half of every box edge (system " + std::to_string(s) + ")");
            if (!(rlist < d.box[k]))
                return set_error(nullptr, ABFE_ERR_CUTOFF_TOO_LARGE, "cutoff + skin must be < box edge");
        }
        if (!finite3(d.pos, 3LL * d.n_atoms) || (d.vel && !finite3(d.vel, 3LL * d.n_atoms)))
            return set_error(nullptr, ABFE_ERR_NONFINITE, "non-finite input coordinate/velocity");
        int nl = 0;
        for (int i = 0; i < d.n_atoms; ++i) {
            if (!(d.mass[i] > 0) || !(d.sigma[i] >= 0) || !(d.epsilon[i] >= 0) || !std::isfinite(d.charge[i]))
                return set_error(nullptr, ABFE_ERR_INVALID_ARG, "bad mass/sigma/epsilon/charge");
            nl += d.is_ligand[i] ? 1 : 0;
        }
        if (nl > COL_MAX) return set_error(nullptr, ABFE_ERR_INVALID_ARG, "more than 1024 ligand atoms");
        if (d.n_excl < 0 || (d.n_excl > 0 && !d.excl) || d.n_bonds < 0 ||
            (d.n_bonds > 0 && (!d.bond_idx || !d.bond_r0 || !d.bond_k)))
            return set_error(nullptr, ABFE_ERR_INVALID_ARG, "bad exclusion/bond arrays");
        for (int k = 0; k < 2 * d.n_excl; ++k)
            if (d.excl[k] < 0 || d.excl[k] >= d.n_atoms)
                return set_error(nullptr, ABFE_ERR_INVALID_ARG, "exclusion index out of range");
        for (int k = 0; k < d.n_excl; ++k)
            if (d.excl[2 * k] == d.excl[2 * k + 1])
                return set_error(nullptr, ABFE_ERR_INVALID_ARG, "self exclusion");
        for (int k = 0; k < 2 * d.n_bonds; ++k)
            if (d.bond_idx[k] < 0 || d.bond_idx[k] >= d.n_atoms)
                return set_error(nullptr, ABFE_ERR_INVALID_ARG, "bond index out of range");
        if (d.n_torsions < 0 || (d.n_torsions > 0 && (!d.torsion_idx || !d.torsion_k ||
                                                      !d.torsion_n || !d.torsion_phi0)))
            return set_error(nullptr, ABFE_ERR_INVALID_ARG, "bad torsion arrays");
        for (int k = 0; k < d.n_torsions; ++k) {
            const int32_t* q = d.torsion_idx + 4 * k;
            for (int a = 0; a < 4; ++a) {
                if (q[a] < 0 || q[a] >= d.n_atoms)
                    return set_error(nullptr, ABFE_ERR_INVALID_ARG, "torsion index out of range");
                for (int b = 0; b < a; ++b)
                    if (q[a] == q[b])
                        return set_error(nullptr, ABFE_ERR_INVALID_ARG, "repeated torsion atom");
            }
            if (d.torsion_n[k] < 1 || d.torsion_n[k] > 6 || !std::isfinite(d.torsion_k[k]) ||
                !std::isfinite(d.torsion_phi0[k]))
                return set_error(nullptr, ABFE_ERR_INVALID_ARG,
                                 "torsion periodicity 1..6 and finite k, phi0");
        }
        if (d.n_alch_waters < 0 || (d.n_alch_waters > 0 && (!d.alch_water_idx || !d.alch_water_dq)))
            return set_error(nullptr, ABFE_ERR_INVALID_ARG, "bad alchemical water arrays");
        for (int k = 0; k < d.n_alch_waters; ++k) {
            const int a = d.alch_water_idx[k];
            if (a < 0 || a >= d.n_atoms || d.is_ligand[a] || !std::isfinite(d.alch_water_dq[k]))
                return set_error(nullptr, ABFE_ERR_INVALID_ARG,
                                 "alchemical water index out of range, a ligand atom, or non-finite dq");
            for (int b = 0; b < k; ++b)
                if (d.alch_water_idx[b] == a)
                    return set_error(nullptr, ABFE_ERR_INVALID_ARG, "repeated alchemical water");
        }
        if (d.n_alch_waters > 0 && p->pme_order > 0)
            return set_error(nullptr, ABFE_ERR_NOT_IMPLEMENTED,
                             "alchemical waters with reciprocal-space Ewald (pme_order > 0)");
        if (d.has_boresch) {
            for (int a = 0; a < 6; ++a) {
                if (d.anchors[a] < 0 || d.anchors[a] >= d.n_atoms)
                    return set_error(nullptr, ABFE_ERR_INVALID_ARG, "Boresch anchor out of range");
                for (int b = 0; b < a; ++b)
                    if (d.anchors[a] == d.anchors[b])
                        return set_error(nullptr, ABFE_ERR_INVALID_ARG, "repeated Boresch anchor");
            }
        }
    }

    c = new abfe_ctx();
    c->prm = *p;
    c->skin_cap = skin_cap;
    c->R = n_replicas;
    c->NS = n_systems;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return set_error(nullptr, ABFE_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return set_error(nullptr, ABFE_ERR_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&c->fork, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    c->tune.group = p->precision == 1 ? 1 : 2;
    c->tune.max_entries = 64;
    c->tune.block_threads = 128;
    c->tune.graph_steps = 0;
    c->tune.skin = p->skin;
    c->tune.prune_skin = std::min(0.5 * p->skin, PRUNE_SKIN_MAX);

    // ---------------------------------------------------------------- systems
    std::vector<float4> h_prm;
    std::vector<dbl4> h_prmd;
    std::vector<unsigned char> h_lig;
    std::vector<int> h_exoff, h_exidx;
    std::vector<int2> h_bond;
    std::vector<float2> h_bondp;
    std::vector<BoreschDev> h_bor;
    std::vector<int4> h_tors;
    std::vector<dbl4> h_torsp;
    std::vector<int> h_aw;
    std::vector<float> h_dq;
    std::vector<double> h_dqd;
    const double sqke = std::sqrt(p->coulomb_k);
    for (int s = 0; s < n_systems; ++s) {
        const abfe_system_desc& d = systems[s];
        const int n = d.n_atoms;
        c->sys_n.push_back(n);
        c->sys_box.push_back({d.box[0], d.box[1], d.box[2]});
        c->sys_atom_off.push_back((int)h_prm.size());
        int nl = 0;
        for (int i = 0; i < n; ++i) {
            h_prm.push_back(make_float4((float)(d.charge[i] * sqke), (float)(0.5 * d.sigma[i]),
                                        (float)(2.0 * std::sqrt(d.epsilon[i])), (float)(1.0 / d.mass[i])));
            h_prmd.push_back(dbl4{d.charge[i], d.sigma[i], d.epsilon[i], 1.0 / d.mass[i]});
            h_lig.push_back(d.is_ligand[i] ? 1 : 0);
            nl += d.is_ligand[i] ? 1 : 0;
        }
        c->sys_nlig.push_back(nl);
        // exclusions: CSR over both directions, sorted, unique
        std::vector<std::vector<int>> ex(n);
        for (int k = 0; k < d.n_excl; ++k) {
            ex[d.excl[2 * k]].push_back(d.excl[2 * k + 1]);
            ex[d.excl[2 * k + 1]].push_back(d.excl[2 * k]);
        }
        c->sys_ex_row.push_back((int)h_exoff.size());
        int nex = 0;
        for (int i = 0; i < n; ++i) {
            std::sort(ex[i].begin(), ex[i].end());
            ex[i].erase(std::unique(ex[i].begin(), ex[i].end()), ex[i].end());
            h_exoff.push_back((int)h_exidx.size());
            for (int j : ex[i]) h_exidx.push_back(j);
            nex += (int)ex[i].size();
        }
        h_exoff.push_back((int)h_exidx.size());
        c->sys_nexcl.push_back(nex / 2);
        c->sys_bond_off.push_back((int)h_bond.size());
        c->sys_nbonds.push_back(d.n_bonds);
        c->max_bonds = std::max(c->max_bonds, d.n_bonds);
        c->sys_ntri.push_back(order_bonds(d, h_bond, h_bondp));
        {
            const size_t base = h_dq.size();
            h_dq.resize(base + n, 0.f);
            h_dqd.resize(base + n, 0.0);
            c->sys_aw_off.push_back((int)h_aw.size());
            c->sys_naw.push_back(d.n_alch_waters);
            c->max_aw = std::max(c->max_aw, d.n_alch_waters);
            for (int k = 0; k < d.n_alch_waters; ++k) {
                const int a = d.alch_water_idx[k];
                h_aw.push_back(a);
                h_dqd[base + a] = d.alch_water_dq[k];
                h_dq[base + a] = (float)(d.alch_water_dq[k] * sqke);
            }
        }
        c->sys_tors_off.push_back((int)h_tors.size());
        c->sys_ntors.push_back(d.n_torsions);
        c->max_tors = std::max(c->max_tors, d.n_torsions);
        for (int k = 0; k < d.n_torsions; ++k) {
            const int32_t* q = d.torsion_idx + 4 * k;
            h_tors.push_back(make_int4(q[0], q[1], q[2], q[3]));
            h_torsp.push_back(dbl4{d.torsion_k[k], (double)d.torsion_n[k], d.torsion_phi0[k], 0.0});
        }
        if (d.has_boresch) {
            BoreschDev B;
            for (int a = 0; a < 6; ++a) B.anc[a] = d.anchors[a];
            B.r0 = d.b_r0;
            B.th0[0] = d.b_theta0[0]; B.th0[1] = d.b_theta0[1];
            B.ph0[0] = d.b_phi0[0]; B.ph0[1] = d.b_phi0[1]; B.ph0[2] = d.b_phi0[2];
            B.kr = d.b_kr; B.kth = d.b_ktheta; B.kph = d.b_kphi;
            c->sys_bor.push_back((int)h_bor.size());
            h_bor.push_back(B);
        } else {
            c->sys_bor.push_back(-1);
        }
    }

    // ---------------------------------------------------------------- replicas
    int cl_off = 0, col_off = 0;
    int64_t atom_off = 0;
    int64_t cap_e = 0, cap_x = 0, cap_items_lig = 64, cap_xrows = 0;
    std::vector<int> h_xrow_cap, h_ritem_cap;   // per replica inner-list regions
    std::vector<int64_t> h_ent_cap, h_xent_cap, h_ienv_cap, h_ilig_cap;   // outer-list regions
    for (int r = 0; r < n_replicas; ++r) {
        const int s = system_of_replica[r];
        const abfe_system_desc& d = systems[s];
        RepDev R{};
        const int n = d.n_atoms, nl = c->sys_nlig[s], ne = n - nl;
        const double V = d.box[0] * d.box[1] * d.box[2];
        const double rho = std::max(n / V, 1.0);
        const double a = std::cbrt(8.0 / rho);
        int ncx = std::max(1, (int)std::floor(d.box[0] / a));
        int ncy = std::max(1, (int)std::floor(d.box[1] / a));
        while ((double)ne / (ncx * ncy) > 0.5 * COL_MAX) { ncx += 1; ncy += 1; }
        R.cl_off = cl_off;
        R.n_cl_cap = (ne + CL - 1) / CL + ncx * ncy + (nl + CL - 1) / CL + 2;
        R.atom_off = (int)atom_off;
        R.n_atoms = n;
        R.n_lig = nl;
        R.sys = s;
        R.sys_atom_off = c->sys_atom_off[s];
        R.sys_ex_off = c->sys_ex_row[s];
        R.col_off = col_off;
        R.ncx = ncx;
        R.ncy = ncy;
        for (int k = 0; k < 3; ++k) R.box[k] = (float)d.box[k];
        R.colw_inv[0] = (float)(ncx / d.box[0]);
        R.colw_inv[1] = (float)(ncy / d.box[1]);
        R.sched = 0; R.state = 0;
        R.lam_q = R.lam_v = 1.f; R.lam_r = 0.f;
        R.dlam_q = R.dlam_v = 1.0; R.dlam_r = 0.0;
        R.sc_A = 0.f; R.sc_dA = (float)(-p->sc_alpha * p->sc_p);
        R.dsc_A = 0.0; R.dsc_dA = -p->sc_alpha * p->sc_p;
        R.bond_off = c->sys_bond_off[s];
        R.n_bonds = c->sys_nbonds[s];
        R.n_bond_tri = c->sys_ntri[s];
        R.boresch = c->sys_bor[s];
        R.kv = 0;
        R.tors_off = c->sys_tors_off[s];
        R.n_tors = c->sys_ntors[s];
        R.aw_off = c->sys_aw_off[s];
        R.n_aw = c->sys_naw[s];
        c->reps_h.push_back(R);
        c->rep_atom_off.push_back(atom_off);
        c->sys_of_rep.push_back(s);
        for (int k = 0; k < R.n_cl_cap; ++k) c->rep_of_cl_h.push_back(r);
        const int64_t epc = est_entries_per_cluster(rho, rlist_cap, R.n_cl_cap);
        cap_e += (int64_t)R.n_cl_cap * epc;
        cap_x += 2LL * c->sys_nexcl[s] + 2LL * R.n_cl_cap + 64;
        h_ent_cap.push_back(std::max<int64_t>((int64_t)R.n_cl_cap * epc, 64));
        h_xent_cap.push_back(2LL * c->sys_nexcl[s] + 2LL * R.n_cl_cap + 64);
        h_ienv_cap.push_back((int64_t)R.n_cl_cap + (int64_t)R.n_cl_cap * epc / 8 + 8);
        c->rep_rho.push_back(rho);
        const int64_t xr_cap = (int64_t)std::ceil(1.25 * (c->sys_nexcl[s] + 8.0 * R.n_cl_cap)) + 64;
        cap_xrows += xr_cap;
        h_xrow_cap.push_back((int)std::min<int64_t>(xr_cap, INT32_MAX));
        h_ritem_cap.push_back((int)std::min<int64_t>(
            2 * ((int64_t)R.n_cl_cap + (int64_t)R.n_cl_cap * epc / 8) + 16, INT32_MAX));
        const int nlc = (nl + CL - 1) / CL;
        c->n_lig_cl += nlc;
        c->max_lig_cl = std::max(c->max_lig_cl, nlc);
        // A ligand cluster's list is a full list (no half-list rule) and its
        // bounding box is as long as its stretch of the chain, so no density
        // estimate bounds it: size the ligand items for every cluster of the
        // replica under every periodic image that can reach (3 per axis whose
        // box edge is below 2 r_list + 3 nm), in items of at most 16 entries.
        int64_t n_img = 1;
        for (int k = 0; k < 3; ++k) n_img *= d.box[k] < 2.0 * rlist_cap + 3.0 ? 3 : 1;
        const int64_t lig_items = nlc ? (int64_t)nlc * (((int64_t)R.n_cl_cap * n_img + 15) / 16 + 1) + 4 : 4;
        cap_items_lig += lig_items;
        h_ilig_cap.push_back(lig_items);
        cl_off += R.n_cl_cap;
        col_off += ncx * ncy + 1;
        atom_off += n;
    }
    while (cl_off % 4) { c->rep_of_cl_h.push_back(-1); ++cl_off; }
    c->C = cl_off;
    c->S = cl_off * CL;
    c->NCOL = col_off;
    c->total_atoms = atom_off;
    const int64_t cap_items_env = (int64_t)c->C + cap_e / 8 + 64;
    if (cap_e > INT32_MAX || cap_x > INT32_MAX || 2 * cap_items_env > INT32_MAX ||
        cap_items_lig > INT32_MAX ||
        cap_xrows > INT32_MAX || c->S > (INT32_MAX / 2) ||
        c->S > (int64_t)ROW_SLOT_MASK + 1) {
        abfe_destroy(c);
        return set_error(nullptr, ABFE_ERR_OUT_OF_MEMORY, "workload exceeds 32-bit list indexing");
    }

    // ---------------------------------------------------------------- device memory
    bool ok = true;
    DevPtrs& P = c->P;
    P.R = c->R;
    P.S = c->S;
    P.C = c->C;
    P.NCOL = c->NCOL;
    c->d_reps = dalloc<RepDev>(c, c->R, ok);
    P.reps = c->d_reps;
    int* d_rep_of_cl = dalloc<int>(c, c->C, ok);
    P.rep_of_cl = d_rep_of_cl;
    P.xq = dalloc<float4>(c, c->S, ok);
    P.v = dalloc<float4>(c, c->S, ok);
    P.se = dalloc<float2>(c, c->S, ok);
    P.orig = dalloc<int>(c, c->S, ok);
    P.xref = dalloc<float4>(c, c->S, ok);
    P.xbuild = dalloc<float4>(c, c->S, ok);
    P.fx = dalloc<long long>(c, c->S, ok);
    P.fy = dalloc<long long>(c, c->S, ok);
    P.fz = dalloc<long long>(c, c->S, ok);
    P.slot_of = dalloc<int>(c, c->total_atoms, ok);
    P.xq_old = dalloc<float4>(c, c->S, ok);
    P.v_old = dalloc<float4>(c, c->S, ok);
    P.orig_old = dalloc<int>(c, c->S, ok);
    P.slot_col = dalloc<int>(c, c->S, ok);
    P.perm = dalloc<int>(c, c->S, ok);
    P.col_atoms = dalloc<int>(c, c->S, ok);
    int* d_col_rep = dalloc<int>(c, c->NCOL, ok);
    P.col_rep = d_col_rep;
    P.col_cnt = dalloc<int>(c, c->NCOL, ok);
    P.col_fill = dalloc<int>(c, c->NCOL, ok);
    P.col_start = dalloc<int>(c, c->NCOL, ok);
    P.col_cl_start = dalloc<int>(c, c->NCOL, ok);
    P.col_ncl = dalloc<int>(c, c->NCOL, ok);
    P.cl_col = dalloc<int>(c, c->C, ok);
    P.bbc = dalloc<float4>(c, c->C, ok);
    P.bbh = dalloc<float4>(c, c->C, ok);
    P.clz = dalloc<float2>(c, c->C, ok);
    float4* d_sys_prm = dalloc<float4>(c, h_prm.size(), ok);
    dbl4* d_sys_prmd = dalloc<dbl4>(c, h_prmd.size(), ok);
    unsigned char* d_sys_lig = dalloc<unsigned char>(c, h_lig.size(), ok);
    int* d_exoff = dalloc<int>(c, h_exoff.size(), ok);
    int* d_exidx = dalloc<int>(c, std::max<size_t>(1, h_exidx.size()), ok);
    int2* d_bond = dalloc<int2>(c, std::max<size_t>(1, h_bond.size()), ok);
    float2* d_bondp = dalloc<float2>(c, std::max<size_t>(1, h_bondp.size()), ok);
    // flattened bond index over all replicas: prefix per replica and, per block
    // of 256 bonds, the replica holding its first bond
    std::vector<int> h_bpref(c->R + 1, 0);
    // the bond kernel's units: a bonded triangle (three bonds) or a single bond
    auto bond_units = [](const RepDev& R) { return R.n_bonds - 2 * R.n_bond_tri; };
    {
        int64_t nb = 0;
        for (int r = 0; r < c->R; ++r) nb += bond_units(c->reps_h[r]);
        if (nb > INT32_MAX - 256) {
            abfe_destroy(c);
            return set_error(nullptr, ABFE_ERR_INVALID_ARG, "more than 2^31 - 257 bonds in all replicas");
        }
    }
    for (int r = 0; r < c->R; ++r) h_bpref[r + 1] = h_bpref[r] + bond_units(c->reps_h[r]);
    c->n_bond_total = h_bpref[c->R];
    std::vector<int> h_bblk((c->n_bond_total + 255) / 256 + 1, 0);
    for (int b = 0, r = 0; b + 1 < (int)h_bblk.size(); ++b) {
        while (h_bpref[r + 1] <= 256 * b) ++r;
        h_bblk[b] = r;
    }
    int* d_bpref = dalloc<int>(c, h_bpref.size(), ok);
    int* d_bblk = dalloc<int>(c, h_bblk.size(), ok);
    BoreschDev* d_bor = dalloc<BoreschDev>(c, std::max<size_t>(1, h_bor.size()), ok);
    int4* d_tors = dalloc<int4>(c, std::max<size_t>(1, h_tors.size()), ok);
    int* d_aw = dalloc<int>(c, std::max<size_t>(1, h_aw.size()), ok);
    float* d_dq = dalloc<float>(c, std::max<size_t>(1, h_dq.size()), ok);
    double* d_dqd = dalloc<double>(c, std::max<size_t>(1, h_dqd.size()), ok);
    dbl4* d_torsp = dalloc<dbl4>(c, std::max<size_t>(1, h_torsp.size()), ok);
    P.sys_prm = d_sys_prm; P.sys_prmd = d_sys_prmd; P.sys_lig = d_sys_lig;
    P.sys_ex_off = d_exoff; P.sys_ex_idx = d_exidx; P.sys_bond = d_bond; P.sys_bond_p = d_bondp;
    P.bond_pref = d_bpref; P.bond_blk_rep = d_bblk; P.n_bond_total = c->n_bond_total;
    P.bor = d_bor;
    P.sys_tors = d_tors;
    P.sys_torsp = d_torsp;
    P.sys_aw = d_aw;
    P.sys_dq = d_dq;
    P.sys_dqd = d_dqd;
    P.has_aw = c->max_aw > 0 ? 1 : 0;
    // outer list: one region per replica
    std::vector<int> h_ent_base(c->R), h_xent_base(c->R), h_ienv_base(c->R), h_ilig_base(c->R);
    std::vector<int> h_ent_c(c->R), h_xent_c(c->R), h_ienv_c(c->R), h_ilig_c(c->R);
    int64_t te = 0, tx = 0, tie = 0, til = 0;
    for (int r = 0; r < c->R; ++r) {
        h_ent_base[r] = (int)std::min<int64_t>(te, INT32_MAX);
        h_xent_base[r] = (int)std::min<int64_t>(tx, INT32_MAX);
        h_ienv_base[r] = (int)std::min<int64_t>(tie, INT32_MAX);
        h_ilig_base[r] = (int)std::min<int64_t>(til, INT32_MAX);
        h_ent_c[r] = (int)std::min<int64_t>(h_ent_cap[r], INT32_MAX);
        h_xent_c[r] = (int)std::min<int64_t>(h_xent_cap[r], INT32_MAX);
        h_ienv_c[r] = (int)std::min<int64_t>(h_ienv_cap[r], INT32_MAX);
        h_ilig_c[r] = (int)std::min<int64_t>(h_ilig_cap[r], INT32_MAX);
        te += h_ent_cap[r];
        tx += h_xent_cap[r];
        tie += h_ienv_cap[r];
        til += h_ilig_cap[r];
    }
    if (te > INT32_MAX || tx > INT32_MAX / GMAX || tie > INT32_MAX || til > INT32_MAX) {
        abfe_destroy(c);
        return set_error(nullptr, ABFE_ERR_OUT_OF_MEMORY, "workload exceeds 32-bit list indexing");
    }
    P.cap_items_env = (int)std::max<int64_t>(tie, 1);
    P.cap_items_lig = (int)std::max<int64_t>(til, 1);
    P.cap_entries = (int)std::max<int64_t>(te, 1);
    P.cap_xentries = (int)std::max<int64_t>(tx, 1);
    int* d_ent_base = dalloc<int>(c, c->R, ok);
    int* d_ent_cap = dalloc<int>(c, c->R, ok);
    int* d_xent_base = dalloc<int>(c, c->R, ok);
    int* d_xent_cap = dalloc<int>(c, c->R, ok);
    int* d_ienv_base = dalloc<int>(c, c->R, ok);
    int* d_ienv_cap = dalloc<int>(c, c->R, ok);
    int* d_ilig_base = dalloc<int>(c, c->R, ok);
    int* d_ilig_cap = dalloc<int>(c, c->R, ok);
    P.ent_base = d_ent_base; P.ent_cap = d_ent_cap;
    P.xent_base = d_xent_base; P.xent_cap = d_xent_cap;
    P.ienv_base = d_ienv_base; P.ienv_cap = d_ienv_cap;
    P.ilig_base = d_ilig_base; P.ilig_cap = d_ilig_cap;
    P.n_entries_r = dalloc<int>(c, c->R, ok);
    P.n_xentries_r = dalloc<int>(c, c->R, ok);
    P.n_items_env_r = dalloc<int>(c, c->R, ok);
    P.n_items_lig_r = dalloc<int>(c, c->R, ok);
    P.ienv_pref = dalloc<int>(c, c->R + 1, ok);
    P.ilig_pref = dalloc<int>(c, c->R + 1, ok);
    P.dispb_r = dalloc<unsigned int>(c, c->R, ok);
    P.bflag = dalloc<int>(c, c->R, ok);
    P.items_env = dalloc<Item>(c, P.cap_items_env, ok);
    P.items_lig = dalloc<Item>(c, P.cap_items_lig, ok);
    P.entries = dalloc<int2>(c, P.cap_entries, ok);
    P.xentries = dalloc<int2>(c, P.cap_xentries, ok);
    P.xmasks = dalloc<unsigned long long>(c, (size_t)P.cap_xentries * GMAX, ok);
    // masked rows and row items: one region per replica
    std::vector<int> h_xrow_base(c->R), h_ritem_base(c->R);
    int64_t xr_tot = 0, ri_tot = 0;
    for (int r = 0; r < c->R; ++r) {
        h_xrow_base[r] = (int)xr_tot;
        h_ritem_base[r] = (int)ri_tot;
        xr_tot += h_xrow_cap[r];
        ri_tot += h_ritem_cap[r];
    }
    if (xr_tot > INT32_MAX || ri_tot > INT32_MAX) {
        abfe_destroy(c);
        return set_error(nullptr, ABFE_ERR_OUT_OF_MEMORY, "workload exceeds 32-bit list indexing");
    }
    P.cap_xrows = (int)std::max<int64_t>(xr_tot, 1);
    P.cap_ritems = (int)std::max<int64_t>(ri_tot, 1);
    P.xrows = dalloc<int2>(c, P.cap_xrows, ok);
    P.ritems = dalloc<RowItem>(c, P.cap_ritems, ok);
    int* d_xrow_base = dalloc<int>(c, c->R, ok);
    int* d_xrow_cap = dalloc<int>(c, c->R, ok);
    int* d_ritem_base = dalloc<int>(c, c->R, ok);
    int* d_ritem_cap = dalloc<int>(c, c->R, ok);
    c->d_row_base = dalloc<unsigned int>(c, c->R, ok);
    c->d_row_cap = dalloc<unsigned int>(c, c->R, ok);
    P.xrow_base = d_xrow_base; P.xrow_cap = d_xrow_cap;
    P.ritem_base = d_ritem_base; P.ritem_cap = d_ritem_cap;
    P.row_base = c->d_row_base; P.row_cap = c->d_row_cap;
    P.n_rows_r = dalloc<unsigned int>(c, c->R, ok);
    P.n_xrows_r = dalloc<int>(c, c->R, ok);
    P.n_ritems_r = dalloc<int>(c, c->R, ok);
    P.ritem_pref = dalloc<int>(c, c->R + 1, ok);
    P.ritem_blk = dalloc<int>(c, (size_t)P.cap_ritems / 256 + 2, ok);
    P.disp_r = dalloc<unsigned int>(c, c->R, ok);
    P.pflag = dalloc<int>(c, c->R, ok);
    P.eacc = dalloc<long long>(c, (size_t)c->R * EA_N, ok);
    P.eb = dalloc<double>(c, c->R, ok);
    P.ukn_lj = dalloc<long long>(c, (size_t)c->R * KV_MAX, ok);
    P.ukn_c = dalloc<long long>(c, (size_t)c->R * 2, ok);
    c->d_sched_state = dalloc<dbl4>(c, (size_t)MAX_SCHED * K_MAX, ok);
    c->d_sched_K = dalloc<int>(c, MAX_SCHED, ok);
    c->d_kv_lam = dalloc<float>(c, (size_t)MAX_SCHED * KV_MAX, ok);
    c->d_kv_A = dalloc<float>(c, (size_t)MAX_SCHED * KV_MAX, ok);
    c->d_kv_dlam = dalloc<double>(c, (size_t)MAX_SCHED * KV_MAX, ok);
    c->d_kv_dA = dalloc<double>(c, (size_t)MAX_SCHED * KV_MAX, ok);
    c->d_sched_sc = dalloc<double2>(c, (size_t)MAX_SCHED * K_MAX, ok);
    c->d_ex = dalloc<int>(c, 4 * (size_t)c->R + 2, ok);
    P.sched_state = c->d_sched_state; P.sched_K = c->d_sched_K;
    P.kv_lam = c->d_kv_lam; P.kv_A = c->d_kv_A; P.kv_dlam = c->d_kv_dlam; P.kv_dA = c->d_kv_dA;
    c->d_energy = dalloc<double>(c, (size_t)c->R * ABFE_N_ENERGY, ok);
    c->d_dudl = dalloc<double>(c, (size_t)c->R * ABFE_N_DUDL, ok);
    c->d_paircnt = dalloc<long long>(c, (size_t)c->R * 2 + 1, ok);
    P.pair_cnt = c->d_paircnt;
    c->d_cnt = dalloc<Counters>(c, 1, ok);
    P.cnt = c->d_cnt;
    c->d_sp = dalloc<StepParams>(c, SP_N, ok);
    P.sp = c->d_sp + SP_ZERO;
    if (!ok) {
        abfe_destroy(c);
        return set_error(nullptr, ABFE_ERR_OUT_OF_MEMORY, "device allocation failed");
    }
    {
        const abfe_status rs = ensure_rows(c, c->tune.prune_skin);
        if (rs != ABFE_OK) {
            g_create_err = c->err;
            abfe_destroy(c);
            return rs;
        }
    }
    P.rc2 = (float)(p->cutoff * p->cutoff);
    P.beta = (float)p->ewald_beta;
    P.nb2l2e = (float)(-p->ewald_beta * p->ewald_beta * 1.4426950408889634);
    P.tbsp = (float)(2.0 * p->ewald_beta / std::sqrt(M_PI));
    P.sqrt_ke = (float)sqke;
    {
        // Coulomb force table on r (smooth there; in r^2 the term in s^{3/2}
        // made the quadratic interpolation lose accuracy at short range), in
        // FP64 from the closed forms: G(r) = erfc(beta r) + (2 beta / sqrt pi) r
        // e^{-beta^2 r^2}, G'(r) = -(4 beta^3 / sqrt pi) r^2 e^{-beta^2 r^2},
        // G''(r) = -(8 beta^3 / sqrt pi) r (1 - beta^2 r^2) e^{-beta^2 r^2}
        const double b = p->ewald_beta, tp = 2.0 / std::sqrt(M_PI);
        const double h = p->cutoff / (EW_NT - 1);
        std::vector<float4> tab(EW_NT);
        for (int j = 0; j < EW_NT; ++j) {
            const double r = j * h;
            const double e = std::exp(-b * b * r * r);
            const double G = std::erfc(b * r) + tp * b * r * e;
            const double G1 = -2.0 * tp * b * b * b * r * r * e;
            const double G2 = -4.0 * tp * b * b * b * r * (1.0 - b * b * r * r) * e;
            tab[j] = make_float4((float)G, (float)(G1 * h), (float)(0.5 * G2 * h * h), 0.f);
        }
        float4* d_tab = dalloc<float4>(c, EW_NT, ok);
        // on the context's stream, after the zero fill queued there by the
        // allocation (a copy on another stream could land before the fill)
        if (!ok ||
            cudaMemcpyAsync(d_tab, tab.data(), sizeof(float4) * EW_NT, cudaMemcpyHostToDevice,
                            c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            abfe_destroy(c);
            return set_error(nullptr, ABFE_ERR_OUT_OF_MEMORY, "Ewald table");
        }
        P.ewtab = d_tab;
        P.ewtab_inv_h = (float)(1.0 / h);
    }
    P.drc2 = p->cutoff * p->cutoff;
    P.dbeta = p->ewald_beta;
    P.dke = p->coulomb_k;
    P.ligand_mode = p->ligand_mode;
    update_grids(c);

    // ---------------------------------------------------------------- uploads
    std::vector<int> h_col_rep(c->NCOL);
    for (int r = 0; r < c->R; ++r)
        for (int k = 0; k < c->reps_h[r].ncx * c->reps_h[r].ncy + 1; ++k)
            h_col_rep[c->reps_h[r].col_off + k] = r;
    std::vector<float4> h_xq(c->S), h_v(c->S);
    std::vector<int> h_orig(c->S, -1), h_clcol(c->C, -1);
    for (int sl = 0; sl < c->S; ++sl) {
        h_xq[sl] = make_float4(DUMMY_FAR + 37.0f * (float)(sl & 1023), DUMMY_FAR + 41.0f * (float)((sl >> 10) & 1023),
                               DUMMY_FAR + 43.0f * (float)((sl >> 20) & 1023), 0.f);
        h_v[sl] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int r = 0; r < c->R; ++r) {
        const RepDev& R = c->reps_h[r];
        const abfe_system_desc& d = systems[R.sys];
        for (int i = 0; i < R.n_atoms; ++i) {
            const int sl = R.cl_off * CL + i;
            const float4 pr = h_prm[R.sys_atom_off + i];
            h_xq[sl] = make_float4((float)d.pos[3 * i], (float)d.pos[3 * i + 1], (float)d.pos[3 * i + 2], pr.x);
            h_v[sl] = d.vel ? make_float4((float)d.vel[3 * i], (float)d.vel[3 * i + 1], (float)d.vel[3 * i + 2], pr.w)
                            : make_float4(0.f, 0.f, 0.f, pr.w);
            h_orig[sl] = i;
        }
    }
    // ---------------------------------------------------------------- PME grids
    c->pme = p->pme_order > 0;
    P.pme = c->pme ? 1 : 0;
    if (c->pme) {
        abfe_status pst = setup_pme(c, systems, n_systems, P);
        if (pst != ABFE_OK) {
            abfe_destroy(c);
            return pst;
        }
    }
    Counters hc{};
    hc.rebuild = 1;
    StepParams hsp[SP_N] = {};
    hsp[SP_ZERO].zero_force = 1;
    hsp[SP_ZERO].c1 = 1.f;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream);
    };
    cudaError_t e = cudaSuccess;
    e = e ? e : up(d_rep_of_cl, c->rep_of_cl_h.data(), sizeof(int) * c->C);
    e = e ? e : up(d_col_rep, h_col_rep.data(), sizeof(int) * c->NCOL);
    e = e ? e : up(P.xq, h_xq.data(), sizeof(float4) * c->S);
    e = e ? e : up(P.xref, h_xq.data(), sizeof(float4) * c->S);
    e = e ? e : up(P.xbuild, h_xq.data(), sizeof(float4) * c->S);
    e = e ? e : up(P.v, h_v.data(), sizeof(float4) * c->S);
    e = e ? e : up(P.orig, h_orig.data(), sizeof(int) * c->S);
    e = e ? e : up(P.cl_col, h_clcol.data(), sizeof(int) * c->C);
    e = e ? e : up(d_sys_prm, h_prm.data(), sizeof(float4) * h_prm.size());
    e = e ? e : up(d_sys_prmd, h_prmd.data(), sizeof(dbl4) * h_prmd.size());
    e = e ? e : up(d_sys_lig, h_lig.data(), h_lig.size());
    e = e ? e : up(d_exoff, h_exoff.data(), sizeof(int) * h_exoff.size());
    if (!h_exidx.empty()) e = e ? e : up(d_exidx, h_exidx.data(), sizeof(int) * h_exidx.size());
    if (!h_bond.empty()) {
        e = e ? e : up(d_bond, h_bond.data(), sizeof(int2) * h_bond.size());
        e = e ? e : up(d_bondp, h_bondp.data(), sizeof(float2) * h_bondp.size());
    }
    e = e ? e : up(d_bpref, h_bpref.data(), sizeof(int) * h_bpref.size());
    e = e ? e : up(d_ent_base, h_ent_base.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ent_cap, h_ent_c.data(), sizeof(int) * c->R);
    e = e ? e : up(d_xent_base, h_xent_base.data(), sizeof(int) * c->R);
    e = e ? e : up(d_xent_cap, h_xent_c.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ienv_base, h_ienv_base.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ienv_cap, h_ienv_c.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ilig_base, h_ilig_base.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ilig_cap, h_ilig_c.data(), sizeof(int) * c->R);
    e = e ? e : up(d_xrow_base, h_xrow_base.data(), sizeof(int) * c->R);
    e = e ? e : up(d_xrow_cap, h_xrow_cap.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ritem_base, h_ritem_base.data(), sizeof(int) * c->R);
    e = e ? e : up(d_ritem_cap, h_ritem_cap.data(), sizeof(int) * c->R);
    e = e ? e : up(d_bblk, h_bblk.data(), sizeof(int) * h_bblk.size());
    if (!h_bor.empty()) e = e ? e : up(d_bor, h_bor.data(), sizeof(BoreschDev) * h_bor.size());
    e = e ? e : up(d_dq, h_dq.data(), sizeof(float) * h_dq.size());
    e = e ? e : up(d_dqd, h_dqd.data(), sizeof(double) * h_dqd.size());
    if (!h_aw.empty()) e = e ? e : up(d_aw, h_aw.data(), sizeof(int) * h_aw.size());
    if (!h_tors.empty()) {
        e = e ? e : up(d_tors, h_tors.data(), sizeof(int4) * h_tors.size());
        e = e ? e : up(d_torsp, h_torsp.data(), sizeof(dbl4) * h_torsp.size());
    }
    e = e ? e : up(c->d_cnt, &hc, sizeof(Counters));
    e = e ? e : up(c->d_sp, hsp, sizeof(hsp));
    e = e ? e : up(c->d_reps, c->reps_h.data(), sizeof(RepDev) * c->R);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        abfe_destroy(c);
        return set_error(nullptr, ABFE_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    // first list build (also validates capacities); a group whose j list does not
    // fit its per-warp buffer (large cutoffs) falls back to one i-cluster per warp
    enqueue_prepare(c, c->stream);
    abfe_status st = check_device(c);
    if (st == ABFE_ERR_LIST_OVERFLOW && c->tune.group > 1) {
        c->tune.group = 1;
        update_grids(c);
        c->force_rebuild = true;
        enqueue_prepare(c, c->stream);
        st = check_device(c);
    }
    if (st != ABFE_OK) {
        g_create_err = c->err;
        abfe_destroy(c);
        return st;
    }
    *out = c;
    return ABFE_OK;
}

void abfe_destroy(abfe_ctx* c) {
    if (!c) return;
    free_all(c);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->fork) cudaStreamDestroy(c->fork);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

namespace {

// softcore A = alpha (1 - lambda_v)^p and dA/dlambda_v (one formula for the
// state table and for replica setup, so both give identical values)
double2 softcore_A(const abfe_params& prm, double lv) {
    const double al = prm.sc_alpha, pp = prm.sc_p;
    return make_double2(al * std::pow(1.0 - lv, pp),
                        -al * pp * (pp == 1.0 ? 1.0 : std::pow(1.0 - lv, pp - 1.0)));
}

// exchange groups from the current replica states (positions by ascending state)
abfe_status upload_exchange(abfe_ctx* c) {
    const int R = c->R;
    std::vector<int> key_of(R, -1);
    std::vector<std::pair<int, int>> keys;
    for (int r = 0; r < R; ++r) {
        const std::pair<int, int> k{c->sys_of_rep[r], c->sched_of_rep[r]};
        int g = -1;
        for (size_t q = 0; q < keys.size(); ++q)
            if (keys[q] == k) g = (int)q;
        if (g < 0) {
            g = (int)keys.size();
            keys.push_back(k);
        }
        key_of[r] = g;
    }
    const int G = (int)keys.size();
    std::vector<int> grp(R), goff(G + 1, 0), slot(R), held(R);
    for (int r = 0; r < R; ++r) goff[key_of[r] + 1] += 1;
    for (int g = 0; g < G; ++g) goff[g + 1] += goff[g];
    std::vector<int> fill(goff.begin(), goff.end() - 1);
    for (int r = 0; r < R; ++r) slot[fill[key_of[r]]++] = r;
    c->ex_unique = true;
    for (int g = 0; g < G; ++g) {
        std::stable_sort(slot.begin() + goff[g], slot.begin() + goff[g + 1],
                         [&](int a, int b) { return c->state_of_rep[a] < c->state_of_rep[b]; });
        for (int p = goff[g]; p < goff[g + 1]; ++p) {
            grp[p] = g;
            held[p] = c->state_of_rep[slot[p]];
            if (p > goff[g] && held[p] == held[p - 1]) c->ex_unique = false;
        }
    }
    std::vector<int> buf(4 * (size_t)R + 2, 0);
    std::copy(grp.begin(), grp.end(), buf.begin());
    std::copy(goff.begin(), goff.end(), buf.begin() + R);
    std::copy(slot.begin(), slot.end(), buf.begin() + 2 * R + 1);
    std::copy(held.begin(), held.end(), buf.begin() + 3 * R + 1);
    CK(cudaMemcpyAsync(c->d_ex, buf.data(), sizeof(int) * buf.size(), cudaMemcpyHostToDevice,
                       c->stream));
    c->ex_goff = goff;
    c->ex_held = held;
    return ABFE_OK;
}

ExchangeDev exchange_dev(abfe_ctx* c) {
    ExchangeDev X{};
    const int R = c->R;
    X.R = R;
    X.grp = c->d_ex;
    X.goff = c->d_ex + R;
    X.slot_rep = c->d_ex + 2 * R + 1;
    X.held = c->d_ex + 3 * R + 1;
    X.n_acc = c->d_ex + 4 * R + 1;
    X.sc = c->d_sched_sc;
    return X;
}

// bring the host copy of the replica states up to date after device exchanges
abfe_status sync_states(abfe_ctx* c) {
    if (!c->reps_dirty) return ABFE_OK;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(c->reps_h.data(), c->d_reps, sizeof(RepDev) * c->R, cudaMemcpyDeviceToHost));
    for (int r = 0; r < c->R; ++r) c->state_of_rep[r] = c->reps_h[r].state;
    c->reps_dirty = false;
    return ABFE_OK;
}

}  // namespace

extern "C" {

abfe_status abfe_set_lambda_schedule(abfe_ctx* c, int32_t id, int32_t K, const double* lr,
                                     const double* lq, const double* lv) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    if (id < 0 || id >= MAX_SCHED || K < 1 || K > K_MAX || !lr || !lq || !lv)
        return set_error(c, ABFE_ERR_INVALID_ARG, "schedule id 0..15, K 1..256, non-NULL arrays");
    SchedHost& S = c->sched[id];
    S.K = K;
    S.lr.assign(lr, lr + K);
    S.lq.assign(lq, lq + K);
    S.lv.assign(lv, lv + K);
    S.kvals.clear();
    S.kvidx.assign(K, 0);
    for (int k = 0; k < K; ++k) {
        if (!(lr[k] >= 0 && lr[k] <= 1 && lq[k] >= 0 && lq[k] <= 1 && lv[k] >= 0 && lv[k] <= 1))
            return set_error(c, ABFE_ERR_INVALID_ARG, "lambda values must lie in [0, 1]");
        int idx = -1;
        for (size_t q = 0; q < S.kvals.size(); ++q)
            if (S.kvals[q] == lv[k]) idx = (int)q;
        if (idx < 0) {
            if ((int)S.kvals.size() >= KV_MAX)
                return set_error(c, ABFE_ERR_INVALID_ARG, "more than 64 distinct lambda_v values");
            idx = (int)S.kvals.size();
            S.kvals.push_back(lv[k]);
        }
        S.kvidx[k] = idx;
    }
    std::vector<dbl4> st(K_MAX, dbl4{0, 0, 0, 0});
    for (int k = 0; k < K; ++k) st[k] = dbl4{lr[k], lq[k], lv[k], (double)S.kvidx[k]};
    std::vector<float> kl(KV_MAX, 0.f), ka(KV_MAX, 0.f);
    std::vector<double> kld(KV_MAX, 0.0), kad(KV_MAX, 0.0);
    for (size_t q = 0; q < S.kvals.size(); ++q) {
        kld[q] = S.kvals[q];
        kad[q] = c->prm.sc_alpha * std::pow(1.0 - S.kvals[q], c->prm.sc_p);
        kl[q] = (float)kld[q];
        ka[q] = (float)kad[q];
    }
    CK(cudaMemcpyAsync(c->d_sched_state + (size_t)id * K_MAX, st.data(), sizeof(dbl4) * K_MAX,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_sched_K + id, &S.K, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_kv_lam + (size_t)id * KV_MAX, kl.data(), sizeof(float) * KV_MAX, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_kv_A + (size_t)id * KV_MAX, ka.data(), sizeof(float) * KV_MAX, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_kv_dlam + (size_t)id * KV_MAX, kld.data(), sizeof(double) * KV_MAX, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_kv_dA + (size_t)id * KV_MAX, kad.data(), sizeof(double) * KV_MAX, cudaMemcpyHostToDevice, c->stream));
    std::vector<double2> sc(K_MAX, make_double2(0.0, 0.0));
    for (int k = 0; k < K; ++k) sc[k] = softcore_A(c->prm, lv[k]);
    CK(cudaMemcpyAsync(c->d_sched_sc + (size_t)id * K_MAX, sc.data(), sizeof(double2) * K_MAX,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->states_set = false;  // replica states must be (re)assigned against the new schedule
    return ABFE_OK;
}

abfe_status abfe_set_replica_states(abfe_ctx* c, const int32_t* sch, const int32_t* state) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    if (!sch || !state) return set_error(c, ABFE_ERR_INVALID_ARG, "NULL arrays");
    for (int r = 0; r < c->R; ++r) {
        if (sch[r] < 0 || sch[r] >= MAX_SCHED || c->sched[sch[r]].K == 0)
            return set_error(c, ABFE_ERR_STATE, "replica uses an unset schedule");
        if (state[r] < 0 || state[r] >= c->sched[sch[r]].K)
            return set_error(c, ABFE_ERR_INVALID_ARG, "state index out of range");
    }
    c->sched_of_rep.assign(sch, sch + c->R);
    c->state_of_rep.assign(state, state + c->R);
    c->reps_dirty = false;
    for (int r = 0; r < c->R; ++r) {
        RepDev& R = c->reps_h[r];
        const SchedHost& S = c->sched[sch[r]];
        const int k = state[r];
        R.sched = sch[r];
        R.state = k;
        R.dlam_r = S.lr[k];
        R.dlam_q = S.lq[k];
        R.dlam_v = S.lv[k];
        R.lam_r = (float)R.dlam_r;
        R.lam_q = (float)R.dlam_q;
        R.lam_v = (float)R.dlam_v;
        const double2 A = softcore_A(c->prm, R.dlam_v);
        R.dsc_A = A.x;
        R.dsc_dA = A.y;
        R.sc_A = (float)R.dsc_A;
        R.sc_dA = (float)R.dsc_dA;
        R.kv = (int)S.kvals.size();
    }
    abfe_status st = upload_reps(c);
    if (st != ABFE_OK) return st;
    if (c->max_aw > 0) launch_aw_refresh(c->P, c->stream);   // alchemical charges at the new states
    st = upload_exchange(c);
    if (st != ABFE_OK) return st;
    CK(cudaStreamSynchronize(c->stream));
    c->states_set = true;
    c->f_valid = false;
    return ABFE_OK;
}

abfe_status abfe_build_neighbor_list(abfe_ctx* c) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    c->force_rebuild = true;
    enqueue_prepare(c, c->stream);
    c->f_valid = false;
    return check_device(c);
}

static abfe_status force_pass(abfe_ctx* c, bool energy) {
    enqueue_prepare(c, c->stream);
    enqueue_forces(c, c->stream, energy);
    return ABFE_OK;
}

abfe_status abfe_compute(abfe_ctx* c, double* h_forces, double* h_energy, double* h_dudl) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    force_pass(c, true);
    DevPtrs P = c->P;
    P.out_energy = c->d_energy;
    P.out_dudl = c->d_dudl;
    launch_finalize(P, c->stream);
    if (h_forces) {
        if (!c->d_atom3) {
            c->d_atom3 = (double*)dev_alloc(c, sizeof(double) * 3 * c->total_atoms);
            if (!c->d_atom3) return set_error(c, ABFE_ERR_OUT_OF_MEMORY, "output buffer");
        }
        launch_scatter_out(c->P, c->stream, 0, c->d_atom3, nullptr, c->n_sm);
    }
    st = check_device(c);
    if (st) return st;
    c->f_valid = true;
    if (h_forces) CK(cudaMemcpy(h_forces, c->d_atom3, sizeof(double) * 3 * c->total_atoms, cudaMemcpyDeviceToHost));
    if (h_energy) CK(cudaMemcpy(h_energy, c->d_energy, sizeof(double) * ABFE_N_ENERGY * c->R, cudaMemcpyDeviceToHost));
    if (h_dudl) CK(cudaMemcpy(h_dudl, c->d_dudl, sizeof(double) * ABFE_N_DUDL * c->R, cudaMemcpyDeviceToHost));
    return ABFE_OK;
}

abfe_status abfe_compute_device(abfe_ctx* c, float* d_forces, double* d_energy, double* d_dudl) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    force_pass(c, true);
    DevPtrs P = c->P;
    P.out_energy = d_energy;
    P.out_dudl = d_dudl;
    if (d_energy || d_dudl) launch_finalize(P, c->stream);
    if (d_forces) launch_scatter_out(c->P, c->stream, 1, nullptr, d_forces, c->n_sm);
    CK(cudaGetLastError());
    c->f_valid = true;
    return ABFE_OK;
}

}  // extern "C"

// One replica-exchange attempt at the end of a step, on the device ("Simulation
// protocol": exchanges among a GPU's windows every 5 ps): the step's closing
// half kick with the current forces, the u_kn rows of every replica at the
// current coordinates (an energy pass), the exchange on those rows, forces for
// the new states, and the half kick with them that opens the next step (the
// integrator fuses the two half kicks of consecutive steps).
static void enqueue_exchange(abfe_ctx* c, cudaStream_t s, bool fork) {
    launch_integrate(with_sp(c, SP_XPOST), s, c->n_sm);
    enqueue_forces(c, s, true, fork);
    cudaMemsetAsync(c->P.ukn_lj, 0, sizeof(long long) * (size_t)c->R * KV_MAX, s);
    cudaMemsetAsync(c->P.ukn_c, 0, sizeof(long long) * (size_t)c->R * 2, s);
    cudaMemsetAsync(&c->d_cnt->lig_next, 0, sizeof(int), s);
    launch_lig_ukn(c->P, s, c->n_sm * 8, c->prm.precision);
    DevPtrs P = c->P;
    P.out_ukn = c->d_ukn;
    P.out_du = c->d_du;
    P.ukn_ld = c->ukn_cap;
    launch_ukn_assemble(P, s, c->prm.kT);
    launch_exchange(c->P, c->d_reps, exchange_dev(c), c->d_ukn, c->ukn_cap, c->ex_seed, s);
    launch_integrate(with_sp(c, SP_ZERO), s, c->n_sm);
    enqueue_forces(c, s, false, fork);
    launch_integrate(with_sp(c, SP_XPRE), s, c->n_sm);
}

// Appends an IF conditional node to the capture of stream s, with its handle
// (default 0), and records `body` into the node's graph through the side stream.
template <class F>
static bool capture_if(abfe_ctx* c, cudaStream_t s, cudaGraphConditionalHandle h, F body) {
    cudaStreamCaptureStatus cs;
    unsigned long long id;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, &ed, &nd) != cudaSuccess) return false;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t cn;
    if (cudaGraphAddNode(&cn, g, deps, ed, nd, &np) != cudaSuccess) return false;
    cudaGraph_t gbody = np.conditional.phGraph_out[0];
    // the side stream only ever records into the body graph: launch nothing on
    // it unless its capture began
    if (cudaStreamBeginCaptureToGraph(c->side, gbody, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return false;
    body(c->side);
    if (cudaStreamEndCapture(c->side, &gbody) != cudaSuccess) return false;
    return cudaStreamUpdateCaptureDependencies(s, &cn, nullptr, 1,
                                               cudaStreamSetCaptureDependencies) == cudaSuccess;
}

extern "C" {

static bool enqueue_step(abfe_ctx* c, cudaStream_t s, int mode) {
    // mode 0: direct launches; 1: capture with conditional rebuild, prune and
    // exchange nodes; 2: predicated capture
    cudaGraphConditionalHandle h_ex = 0;
    prof_rec(c, c->ev_int, true, s);
    launch_integrate(with_sp(c, SP_STEP), s, c->n_sm);
    prof_rec(c, c->ev_int, false, s);
    if (mode == 1) {
        cudaStreamCaptureStatus cs;
        unsigned long long id;
        cudaGraph_t g;
        if (cudaStreamGetCaptureInfo(s, &cs, &id, &g, nullptr, nullptr, nullptr) != cudaSuccess)
            return false;
        cudaGraphConditionalHandle h_rb, h_pr;
        if (cudaGraphConditionalHandleCreate(&h_rb, g, 0, 0) != cudaSuccess) return false;
        if (cudaGraphConditionalHandleCreate(&h_pr, g, 0, 0) != cudaSuccess) return false;
        if (c->ex_every > 0 && cudaGraphConditionalHandleCreate(&h_ex, g, 0, 0) != cudaSuccess)
            return false;
        launch_step_end(c->P, s, 1, 0, 0, h_rb, h_pr, h_ex, 1);
        if (!capture_if(c, s, h_rb, [&](cudaStream_t b) {
                launch_rebuild(c->P, b, c->n_sm);
                launch_list_build(c->P, b, c->max_lig_cl);
            }))
            return false;
        if (!capture_if(c, s, h_pr, [&](cudaStream_t b) { launch_prune(c->P, b, c->n_sm); }))
            return false;
    } else {
        // the predicated form has no place for an exchange: only direct launches do
        if (mode == 2 && c->ex_every > 0) return false;
        launch_step_end(c->P, s, 1, 0, 0, 0, 0, 0, 0);
        launch_rebuild(c->P, s, c->n_sm);
        launch_list_build(c->P, s, c->max_lig_cl);
        launch_prune(c->P, s, c->n_sm);
    }
    enqueue_forces(c, s, false);
    if (c->ex_every > 0) {
        if (mode == 1) {
            if (!capture_if(c, s, h_ex, [&](cudaStream_t b) { enqueue_exchange(c, b, false); }))
                return false;
        } else {
            c->dev_step += 1;
            if (c->dev_step % (unsigned long long)c->ex_every == 0ull) enqueue_exchange(c, s, true);
        }
    } else if (mode == 0) {
        c->dev_step += 1;
    }
    return true;
}

static abfe_status build_graph(abfe_ctx* c, int nsteps) {
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    for (int mode : {1, 2}) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        bool ok = true;
        for (int i = 0; i < nsteps && ok; ++i) ok = enqueue_step(c, c->stream, mode);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (!ok && e == cudaSuccess) e = cudaErrorStreamCaptureInvalidated;
        if (e == cudaSuccess && g) e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) {
            c->g_steps = nsteps;
            c->g_mode = mode;
            c->g_prof = c->prof_max > 0;
            return ABFE_OK;
        }
        cudaGetLastError();
        c->gexec = nullptr;
    }
    return set_error(c, ABFE_ERR_CUDA, "CUDA graph capture of the step loop failed");
}

abfe_status abfe_step(abfe_ctx* c, int32_t n_steps, double dt, double gamma, uint64_t seed) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    if (n_steps < 0 || !(dt > 0) || !(gamma >= 0))
        return set_error(c, ABFE_ERR_INVALID_ARG, "n_steps >= 0, dt > 0, gamma >= 0");
    if (n_steps == 0) return ABFE_OK;
    if (!c->f_valid) {
        force_pass(c, false);
        c->f_valid = true;
    }
    const double c1 = std::exp(-gamma * dt);
    StepParams sp[SP_N] = {};
    sp[SP_PRE].kick = (float)(-0.5 * dt);
    sp[SP_PRE].c1 = 1.f;
    sp[SP_STEP].kick = (float)dt;
    sp[SP_STEP].half_dt = (float)(0.5 * dt);
    sp[SP_STEP].c1 = (float)c1;
    sp[SP_STEP].c2 = (float)std::sqrt(std::max(0.0, 1.0 - c1 * c1) * c->prm.kT);
    sp[SP_STEP].seed = seed;
    sp[SP_STEP].drift = 1;
    sp[SP_STEP].zero_force = 1;
    sp[SP_POST].kick = (float)(0.5 * dt);
    sp[SP_POST].c1 = 1.f;
    sp[SP_ZERO].c1 = 1.f;
    sp[SP_ZERO].zero_force = 1;
    sp[SP_XPOST].kick = (float)(0.5 * dt);     // closing half kick before an exchange
    sp[SP_XPOST].c1 = 1.f;
    sp[SP_XPOST].zero_force = 1;
    sp[SP_XPRE].kick = (float)(-0.5 * dt);     // reopening after it, with the new forces
    sp[SP_XPRE].c1 = 1.f;
    CK(cudaMemcpyAsync(c->d_sp, sp, sizeof(sp), cudaMemcpyHostToDevice, c->stream));
    if (c->ex_every > 0) {
        abfe_status es = ensure_ukn(c, max_K(c));
        if (es) return es;
    }
    launch_integrate(with_sp(c, SP_PRE), c->stream, c->n_sm);
    int done = 0;
    const int gs = c->tune.graph_steps;
    if (gs > 0 && n_steps >= gs) {
        if (!c->gexec || c->g_steps != gs || c->g_prof != (c->prof_max > 0)) {
            st = build_graph(c, gs);
            if (st) return st;
        }
        while (n_steps - done >= gs) {
            CK(cudaGraphLaunch(c->gexec, c->stream));
            done += gs;
            c->dev_step += (unsigned long long)gs;
        }
    }
    while (done < n_steps) {
        enqueue_step(c, c->stream, 0);
        ++done;
    }
    launch_integrate(with_sp(c, SP_POST), c->stream, c->n_sm);
    st = check_device(c);
    c->steps_done += n_steps;
    if (c->ex_every > 0) c->reps_dirty = true;   // states may have moved on the device
    return st;
}

}  // extern "C"

namespace {

int max_K(abfe_ctx* c) {
    int kmax = 0;
    for (int r = 0; r < c->R; ++r) kmax = std::max(kmax, c->sched[c->sched_of_rep[r]].K);
    return kmax;
}

abfe_status ensure_ukn(abfe_ctx* c, int ld) {
    if (ld > c->ukn_cap) {
        c->d_ukn = (double*)dev_alloc(c, sizeof(double) * (size_t)c->R * ld);
        c->d_du = (double*)dev_alloc(c, sizeof(double) * (size_t)c->R * ld);
        if (!c->d_ukn || !c->d_du) return set_error(c, ABFE_ERR_OUT_OF_MEMORY, "u_kn buffers");
        c->ukn_cap = ld;
    }
    return ABFE_OK;
}

// u_kn rows (reduced), their lambda parts, dU/dlambda and energies of every
// replica at the current coordinates, into the device buffers (stream order)
abfe_status enqueue_ukn(abfe_ctx* c, int ld) {
    abfe_status st = ensure_ukn(c, ld);
    if (st) return st;
    force_pass(c, true);
    CK(cudaMemsetAsync(c->P.ukn_lj, 0, sizeof(long long) * (size_t)c->R * KV_MAX, c->stream));
    CK(cudaMemsetAsync(c->P.ukn_c, 0, sizeof(long long) * (size_t)c->R * 2, c->stream));
    CK(cudaMemsetAsync(&c->d_cnt->lig_next, 0, sizeof(int), c->stream));
    launch_lig_ukn(c->P, c->stream, c->n_sm * 8, c->prm.precision);
    DevPtrs P = c->P;
    P.out_ukn = c->d_ukn;
    P.out_du = c->d_du;
    P.ukn_ld = ld;
    P.out_dudl = c->d_dudl;
    P.out_energy = c->d_energy;
    launch_ukn_assemble(P, c->stream, c->prm.kT);
    launch_finalize(P, c->stream);
    return ABFE_OK;
}

}  // namespace

extern "C" {

abfe_status abfe_eval_ukn(abfe_ctx* c, double* h_ukn, double* h_du, int32_t ld, double* h_dudl) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    if (!h_ukn || ld < max_K(c)) return set_error(c, ABFE_ERR_INVALID_ARG, "h_ukn NULL or ld < K");
    st = enqueue_ukn(c, ld);
    if (st) return st;
    st = check_device(c);
    if (st) return st;
    c->f_valid = true;
    CK(cudaMemcpy(h_ukn, c->d_ukn, sizeof(double) * (size_t)c->R * ld, cudaMemcpyDeviceToHost));
    if (h_du) CK(cudaMemcpy(h_du, c->d_du, sizeof(double) * (size_t)c->R * ld, cudaMemcpyDeviceToHost));
    if (h_dudl) CK(cudaMemcpy(h_dudl, c->d_dudl, sizeof(double) * (size_t)c->R * ABFE_N_DUDL, cudaMemcpyDeviceToHost));
    return ABFE_OK;
}

abfe_status abfe_replica_exchange(abfe_ctx* c, uint64_t seed, const double* h_ukn, int32_t ld,
                                  double* h_ukn_out, int32_t* h_state, int32_t* h_n_accepted) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    if (ld < max_K(c)) return set_error(c, ABFE_ERR_INVALID_ARG, "ld < K");
    if (!c->ex_unique)
        return set_error(c, ABFE_ERR_STATE,
                         "replica exchange needs distinct states within each (system, schedule) group");
    if (h_ukn) {
        for (size_t i = 0; i < (size_t)c->R * ld; ++i) {
            const int k = (int)(i % ld);
            if (k < c->sched[c->sched_of_rep[i / ld]].K && !std::isfinite(h_ukn[i]))
                return set_error(c, ABFE_ERR_NONFINITE, "non-finite u_kn entry");
        }
        st = ensure_ukn(c, ld);
        if (st) return st;
        CK(cudaMemcpyAsync(c->d_ukn, h_ukn, sizeof(double) * (size_t)c->R * ld,
                           cudaMemcpyHostToDevice, c->stream));
    } else {
        st = enqueue_ukn(c, ld);
        if (st) return st;
    }
    const ExchangeDev X = exchange_dev(c);
    launch_exchange(c->P, c->d_reps, X, c->d_ukn, ld, seed, c->stream);
    int acc = 0;
    CK(cudaMemcpyAsync(&acc, X.n_acc, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    st = check_device(c);
    if (st) return st;
    c->reps_dirty = true;
    c->f_valid = false;   // forces belong to the old states
    if (h_ukn_out && !h_ukn)
        CK(cudaMemcpy(h_ukn_out, c->d_ukn, sizeof(double) * (size_t)c->R * ld, cudaMemcpyDeviceToHost));
    if (h_n_accepted) *h_n_accepted = acc;
    if (h_state) {
        st = sync_states(c);
        if (st) return st;
        std::copy(c->state_of_rep.begin(), c->state_of_rep.end(), h_state);
    }
    return ABFE_OK;
}

abfe_status abfe_get_replica_states(abfe_ctx* c, int32_t* h_state) {
    if (!c || !h_state) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    st = sync_states(c);
    if (st) return st;
    std::copy(c->state_of_rep.begin(), c->state_of_rep.end(), h_state);
    return ABFE_OK;
}

abfe_status abfe_set_exchange(abfe_ctx* c, int32_t every_steps, uint64_t seed) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    if (every_steps < 0) return set_error(c, ABFE_ERR_INVALID_ARG, "every_steps >= 0");
    if (every_steps > 0) {
        abfe_status st = need_states(c);
        if (st) return st;
        if (!c->ex_unique)
            return set_error(c, ABFE_ERR_STATE,
                             "replica exchange needs distinct states within each (system, schedule) group");
        st = ensure_ukn(c, max_K(c));
        if (st) return st;
    }
    c->ex_every = every_steps;
    c->ex_seed = seed;
    c->P.ex_every = every_steps;
    c->P.ex_seed = seed;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return ABFE_OK;
}

static abfe_status io_atoms(abfe_ctx* c, int what, double* out, const double* in) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    if (!out && !in) return set_error(c, ABFE_ERR_INVALID_ARG, "NULL array");
    if (!c->d_atom3) {
        c->d_atom3 = (double*)dev_alloc(c, sizeof(double) * 3 * c->total_atoms);
        if (!c->d_atom3) return set_error(c, ABFE_ERR_OUT_OF_MEMORY, "io buffer");
    }
    const size_t bytes = sizeof(double) * 3 * c->total_atoms;
    if (in) {
        if (!finite3(in, 3 * c->total_atoms)) return set_error(c, ABFE_ERR_NONFINITE, "non-finite input");
        CK(cudaMemcpyAsync(c->d_atom3, in, bytes, cudaMemcpyHostToDevice, c->stream));
        launch_gather_in(c->P, c->stream, what, c->d_atom3, c->n_sm);
        if (what == 2) {
            c->force_rebuild = true;
            c->f_valid = false;
        }
        CK(cudaStreamSynchronize(c->stream));
        return check_device(c);
    }
    launch_scatter_out(c->P, c->stream, what, c->d_atom3, nullptr, c->n_sm);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(out, c->d_atom3, bytes, cudaMemcpyDeviceToHost));
    return check_device(c);
}

abfe_status abfe_get_positions(abfe_ctx* c, double* h) { return io_atoms(c, 2, h, nullptr); }
abfe_status abfe_set_positions(abfe_ctx* c, const double* h) { return io_atoms(c, 2, nullptr, h); }
abfe_status abfe_get_velocities(abfe_ctx* c, double* h) { return io_atoms(c, 3, h, nullptr); }
abfe_status abfe_set_velocities(abfe_ctx* c, const double* h) { return io_atoms(c, 3, nullptr, h); }

abfe_status abfe_count_pairs(abfe_ctx* c, int64_t* h_counts, int32_t* h_atom) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    if (!h_counts) return set_error(c, ABFE_ERR_INVALID_ARG, "h_counts NULL");
    enqueue_prepare(c, c->stream);
    c->f_valid = false;
    if (h_atom && !c->d_atomcnt) {
        c->d_atomcnt = (int*)dev_alloc(c, sizeof(int) * c->S);
        if (!c->d_atomcnt) return set_error(c, ABFE_ERR_OUT_OF_MEMORY, "count buffer");
    }
    CK(cudaMemsetAsync(c->d_paircnt, 0, sizeof(long long) * (2 * c->R + 1), c->stream));
    if (h_atom) CK(cudaMemsetAsync(c->d_atomcnt, 0, sizeof(int) * c->S, c->stream));
    DevPtrs P = c->P;
    P.atom_cnt = h_atom ? c->d_atomcnt : nullptr;
    launch_count_pairs(P, c->stream, c->n_sm * 8, 128);
    abfe_status st = check_device(c);
    if (st) return st;
    CK(cudaMemcpy(h_counts, c->d_paircnt, sizeof(long long) * 2 * c->R, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&c->lane_groups, c->d_paircnt + 2 * c->R, sizeof(long long), cudaMemcpyDeviceToHost));
    if (h_atom) {
        std::vector<int> cnt(c->S), orig(c->S);
        CK(cudaMemcpy(cnt.data(), c->d_atomcnt, sizeof(int) * c->S, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(orig.data(), c->P.orig, sizeof(int) * c->S, cudaMemcpyDeviceToHost));
        std::fill(h_atom, h_atom + c->total_atoms, 0);
        for (int s = 0; s < c->S; ++s) {
            if (orig[s] < 0) continue;
            const int r = c->rep_of_cl_h[s >> 3];
            h_atom[c->rep_atom_off[r] + orig[s]] = cnt[s];
        }
    }
    return ABFE_OK;
}

abfe_status abfe_set_tuning(abfe_ctx* c, const abfe_tuning* t) {
    if (!c || !t) return ABFE_ERR_INVALID_ARG;
    if (!(t->group == 1 || t->group == 2 || t->group == 4) || t->max_entries < 16 ||
        t->max_entries > 512 || t->block_threads < 64 || t->block_threads > 256 ||
        (t->block_threads % 32) || t->graph_steps < 0 || !(t->skin >= 0) ||
        t->skin > c->skin_cap + 1e-12 || !(t->prune_skin >= 0) || t->prune_skin > t->skin ||
        t->prune_skin > PRUNE_SKIN_MAX + 1e-12 || t->reserved0 != 0 || t->reserved1 != 0)
        return set_error(c, ABFE_ERR_INVALID_ARG,
                         "group 1/2/4, max_entries 16..512, block_threads 64..256 (x32), "
                         "graph_steps >= 0, 0 <= skin <= " + std::to_string(c->skin_cap) +
                         ", 0 <= prune_skin <= min(skin, 0.15), reserved fields 0");
    const bool relist = t->group != c->tune.group || t->max_entries != c->tune.max_entries ||
                        t->skin != c->tune.skin || t->prune_skin != c->tune.prune_skin;
    const bool regraph = relist || t->block_threads != c->tune.block_threads;
    if (t->prune_skin > c->rows_skin) {
        const abfe_status rs = ensure_rows(c, t->prune_skin);
        if (rs != ABFE_OK) return rs;
    }
    c->tune = *t;
    if (c->prm.precision == 1) c->tune.group = 1;
    update_grids(c);
    if (relist) {
        c->force_rebuild = true;
        c->f_valid = false;
    }
    if (regraph && c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return ABFE_OK;
}

abfe_status abfe_get_tuning(abfe_ctx* c, abfe_tuning* t) {
    if (!c || !t) return ABFE_ERR_INVALID_ARG;
    *t = c->tune;
    return ABFE_OK;
}

abfe_status abfe_get_stats(abfe_ctx* c, abfe_stats* s) {
    if (!c || !s) return ABFE_ERR_INVALID_ARG;
    Counters h;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(&h, c->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost));
    s->n_items_env = h.n_items_env;
    s->n_items_lig = h.n_items_lig;
    s->n_entries = h.n_entries;
    s->n_xentries = h.n_xentries;
    s->n_rebuilds = h.n_rebuilds;
    s->steps_done = c->steps_done;
    s->slots = c->S;
    s->clusters = c->C;
    s->device_bytes = c->device_bytes;
    s->env_lane_groups = c->lane_groups;
    s->n_prunes = h.n_prunes;
    s->n_rows = h.n_rows;
    s->n_xrows = h.n_xrows;
    s->n_exchange_attempts = (int64_t)h.ex_attempt;
    s->n_exchange_accepted = h.ex_accepted;
    s->n_window_rebuilds = (int64_t)h.n_win_rebuilds;
    s->n_window_prunes = (int64_t)h.n_win_prunes;
    return ABFE_OK;
}

abfe_status abfe_set_profiling(abfe_ctx* c, int32_t max_launches) {
    if (!c || max_launches < 0) return ABFE_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->stream));
    for (EventPool* ep : {&c->ev_env, &c->ev_lig, &c->ev_int, &c->ev_build, &c->ev_prune}) {
        for (auto e : ep->a) cudaEventDestroy(e);
        for (auto e : ep->b) cudaEventDestroy(e);
        ep->a.assign(max_launches, nullptr);
        ep->b.assign(max_launches, nullptr);
        for (int i = 0; i < max_launches; ++i) {
            CK(cudaEventCreate(&ep->a[i]));
            CK(cudaEventCreate(&ep->b[i]));
        }
        ep->used = 0;
    }
    c->prof_max = max_launches;
    if (c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; }
    return ABFE_OK;
}

abfe_status abfe_get_profile(abfe_ctx* c, abfe_profile* out) {
    if (!c || !out) return ABFE_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->stream));
    auto sum = [&](EventPool& ep, double& ms, int64_t& n) -> abfe_status {
        ms = 0.0;
        n = ep.used;
        for (int i = 0; i < ep.used; ++i) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ep.a[i], ep.b[i]));
            ms += t;
        }
        return ABFE_OK;
    };
    abfe_status st = sum(c->ev_env, out->env_ms, out->env_launches);
    if (!st) st = sum(c->ev_lig, out->lig_ms, out->lig_launches);
    if (!st) st = sum(c->ev_int, out->integrate_ms, out->integrate_launches);
    if (!st) st = sum(c->ev_build, out->build_ms, out->build_launches);
    if (!st) st = sum(c->ev_prune, out->prune_ms, out->prune_launches);
    return st;
}

}  // extern "C"

namespace {

// The dynamic state of a context in original atom order: positions,
// velocities, positions at the last prune and at the last outer list build, the
// Langevin step counter and the displacement accumulator. Restoring it rebuilds
// the outer list from the saved build positions and prunes at the saved prune
// positions (the builder and the prune are deterministic, so slot order and
// lists are those of the original run) and then puts the state back, so the
// trajectory continues bit for bit.
struct HostState {
    std::vector<double> x, v, xp, xb;
    unsigned long long step = 0;
    unsigned int maxdisp2 = 0;
    int64_t steps_done = 0;
    unsigned long long ex_attempt = 0;
    long long ex_accepted = 0;
};

abfe_status save_state(abfe_ctx* c, HostState& h) {
    const size_t n3 = 3 * (size_t)c->total_atoms;
    h.x.resize(n3);
    h.v.resize(n3);
    h.xp.resize(n3);
    h.xb.resize(n3);
    abfe_status st = abfe_get_positions(c, h.x.data());
    if (!st) st = abfe_get_velocities(c, h.v.data());
    if (st) return st;
    launch_scatter_out(c->P, c->stream, 4, c->d_atom3, nullptr, c->n_sm);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(h.xp.data(), c->d_atom3, sizeof(double) * n3, cudaMemcpyDeviceToHost));
    launch_scatter_out(c->P, c->stream, 5, c->d_atom3, nullptr, c->n_sm);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(h.xb.data(), c->d_atom3, sizeof(double) * n3, cudaMemcpyDeviceToHost));
    Counters hc;
    CK(cudaMemcpy(&hc, c->d_cnt, sizeof(Counters), cudaMemcpyDeviceToHost));
    h.step = hc.step;
    h.maxdisp2 = hc.maxdisp2;
    h.steps_done = c->steps_done;
    h.ex_attempt = hc.ex_attempt;
    h.ex_accepted = hc.ex_accepted;
    return ABFE_OK;
}

abfe_status restore_state(abfe_ctx* c, const HostState& h) {
    abfe_status st = abfe_set_positions(c, h.xb.data());
    if (st) return st;
    c->force_rebuild = true;
    enqueue_prepare(c, c->stream);                  // outer list (and a prune) at the build positions
    st = check_device(c);
    if (st) return st;
    st = abfe_set_positions(c, h.xp.data());
    if (st) return st;
    c->force_rebuild = false;
    c->force_prune = true;
    enqueue_prepare(c, c->stream);                  // inner list at the prune positions
    st = check_device(c);
    if (st) return st;
    st = abfe_set_positions(c, h.x.data());
    if (st) return st;
    c->force_rebuild = false;
    c->force_prune = false;
    st = abfe_set_velocities(c, h.v.data());
    if (st) return st;
    CK(cudaMemcpyAsync(&c->d_cnt->step, &h.step, sizeof h.step, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(&c->d_cnt->maxdisp2, &h.maxdisp2, sizeof h.maxdisp2, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaMemcpyAsync(&c->d_cnt->ex_attempt, &h.ex_attempt, sizeof h.ex_attempt,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(&c->d_cnt->ex_accepted, &h.ex_accepted, sizeof h.ex_accepted,
                       cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->dev_step = h.step;
    c->steps_done = h.steps_done;
    c->f_valid = false;
    return ABFE_OK;
}

}  // namespace

extern "C" {

abfe_status abfe_autotune(abfe_ctx* c, const char* cache_path, int32_t reps) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    if (reps < 1) reps = 3;
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, c->device));
    // key: device, workload size and shape (atoms, windows, mean density,
    // smallest and largest box edge), cutoff, skins, precision
    double vol = 0.0, emin = 1e30, emax = 0.0;
    for (int r = 0; r < c->R; ++r) {
        const std::array<double, 3>& b = c->sys_box[c->sys_of_rep[r]];
        vol += b[0] * b[1] * b[2];
        for (int k = 0; k < 3; ++k) { emin = std::min(emin, b[k]); emax = std::max(emax, b[k]); }
    }
    char key[512];
    snprintf(key, sizeof key,
             "%s|atoms=%lld|R=%d|rho=%.2f|edge=%.3f-%.3f|rc=%.4f|skin=%.4f/%.4f|prec=%d", prop.name,
             (long long)c->total_atoms, c->R, c->total_atoms / std::max(vol, 1e-30), emin, emax,
             c->prm.cutoff, c->tune.skin, c->tune.prune_skin, c->prm.precision);
    abfe_tuning best = c->tune;
    // the sweep rebuilds and prunes the lists for every candidate: it runs from a
    // saved state that is put back afterwards (lists rebuilt from the saved build
    // and prune positions), so the trajectory does not depend on the sweep (nor
    // on whether the tuning came from the cache)
    HostState saved;
    st = save_state(c, saved);
    if (st) return st;
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            const std::string k = std::string("{\"key\": \"") + key + "\"";
            if (line.compare(0, k.size(), k) != 0) continue;
            int g = 0, me = 0, bt = 0;
            const char* q = line.c_str() + k.size();
            if (sscanf(q, ", \"group\": %d, \"max_entries\": %d, \"block_threads\": %d",
                       &g, &me, &bt) == 3) {
                best.group = g; best.max_entries = me; best.block_threads = bt;
                st = abfe_set_tuning(c, &best);
                if (st) return st;
                return restore_state(c, saved);
            }
        }
    }
    cudaEvent_t e0, e1, e2;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventCreate(&e2));
    const int saved_prof = c->prof_max;
    c->prof_max = 0;
    // one candidate: rebuild and prune its lists, then `reps` timed (prune,
    // environment pass) pairs; returns the mean prune and pass times
    auto trial = [&](const abfe_tuning& t, float& prune_ms, float& env_ms) -> bool {
        if (abfe_set_tuning(c, &t) != ABFE_OK) return false;
        enqueue_prepare(c, c->stream);
        if (check_device(c) != ABFE_OK) return false;
        prune_ms = env_ms = 0.f;
        for (int i = 0; i <= reps; ++i) {    // the first round warms up
            c->force_prune = true;
            launch_integrate(with_sp(c, SP_ZERO), c->stream, c->n_sm);
            launch_step_end(c->P, c->stream, 0, 0, 1, 0, 0, 0, 0);
            cudaEventRecord(e0, c->stream);
            launch_prune(c->P, c->stream, c->n_sm);
            cudaEventRecord(e1, c->stream);
            launch_env_forces(c->P, c->stream, false, c->prm.precision, c->env_grid,
                              t.block_threads);
            cudaEventRecord(e2, c->stream);
            cudaEventSynchronize(e2);
            c->force_prune = false;
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, e0, e1);
            cudaEventElapsedTime(&b, e1, e2);
            if (i > 0) { prune_ms += a / reps; env_ms += b / reps; }
        }
        return check_device(c) == ABFE_OK;
    };
    // stage 1: outer-list grouping and work-item length, by pass time plus a
    // quarter of the prune time (about one prune in four steps); stage 2: the
    // pair kernel's block size, by pass time
    std::vector<int> groups = c->prm.precision == 1 ? std::vector<int>{1} : std::vector<int>{1, 2, 4};
    const int mes[] = {32, 64, 128, 512};
    float best_cost = 1e30f, best_env = 1e30f;
    for (int g : groups)
        for (int me : mes) {
            abfe_tuning t = c->tune;
            t.group = g;
            t.max_entries = me;
            float pm = 0.f, em = 0.f;
            if (!trial(t, pm, em)) continue;
            const float cost = em + 0.25f * pm;
            if (cost < best_cost) { best_cost = cost; best = t; best_env = em; }
        }
    const abfe_tuning base = best;
    for (int bt : {128, 256}) {
        if (bt == base.block_threads) continue;
        abfe_tuning t = base;
        t.block_threads = bt;
        float pm = 0.f, em = 0.f;
        if (!trial(t, pm, em)) continue;
        if (em < best_env) { best_env = em; best = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    c->prof_max = saved_prof;
    st = abfe_set_tuning(c, &best);
    if (st) return st;
    st = restore_state(c, saved);
    if (st) return st;
    if (cache_path) {
        std::ofstream o(cache_path, std::ios::app);
        o << "{\"key\": \"" << key << "\", \"group\": " << best.group << ", \"max_entries\": "
          << best.max_entries << ", \"block_threads\": " << best.block_threads
          << ", \"env_ms\": " << best_env << "}\n";
    }
    return ABFE_OK;
}

abfe_status abfe_autotune_cadence(abfe_ctx* c, double dt, double gamma, uint64_t seed,
                                  int32_t n_steps) {
    if (!c) return ABFE_ERR_INVALID_ARG;
    abfe_status st = need_states(c);
    if (st) return st;
    if (n_steps < 8) n_steps = 48;
    // everything runs from a saved state that is restored afterwards: the
    // trajectory (and its rebuild cadence) is the one without the tuner
    HostState saved;
    st = save_state(c, saved);
    if (st) return st;
    const int saved_ex = c->ex_every;              // no exchanges while tuning
    c->ex_every = 0;
    c->P.ex_every = 0;
    const abfe_tuning base = c->tune;
    const int saved_prof = c->prof_max;
    c->prof_max = 0;
    // (1) growth of the largest displacement of any atom with the number of
    // steps, D(n), from an outer build at step 0 (the largest skin, so that no
    // rebuild resets the reference early)
    std::vector<double> D(1, 0.0);
    {
        abfe_tuning t = base;
        t.graph_steps = 0;
        t.skin = c->skin_cap;
        t.prune_skin = PRUNE_SKIN_MAX;
        st = abfe_set_tuning(c, &t);
        if (!st) st = abfe_build_neighbor_list(c);
        for (int n = 1; !st && n <= n_steps; ++n) {
            st = abfe_step(c, 1, dt, gamma, seed + (uint64_t)n);
            if (st) break;
            unsigned int b = 0u;
            CK(cudaMemcpy(&b, &c->d_cnt->last_dispb2, sizeof b, cudaMemcpyDeviceToHost));
            float f;
            memcpy(&f, &b, sizeof f);
            D.push_back(std::sqrt((double)f));
            if (D.back() > 0.5 * c->skin_cap) break;   // the next step rebuilds
        }
    }
    // steps until an atom has moved more than h: the first n with D(n) > h;
    // past the measured range, the last measured growth per step continues
    auto steps_to = [&](double h) -> double {
        for (size_t n = 1; n < D.size(); ++n)
            if (D[n] > h) return (double)n;
        const size_t m = D.size() - 1;
        const double rate = m >= 1 ? std::max(D[m] - D[m > 4 ? m - 4 : 0], 1e-9) /
                                         (double)(m > 4 ? 4 : m)
                                   : 1e-9;
        return (double)m + (h - D[m]) / rate;
    };
    // (2) costs, each from a forced build / prune and one force pass: the outer
    // build B(skin), the prune P(skin, prune_skin), the pair pass E(prune_skin)
    const double cand[] = {0.1, 0.15, 0.2, 0.25, 0.3};
    const double pcand[] = {0.02, 0.04, 0.06, 0.1, 0.15};
    cudaEvent_t e0, e1, e2;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventCreate(&e2));
    auto timed = [&](bool rebuild, float& build_ms, float& prune_ms, float& env_ms) -> bool {
        launch_integrate(with_sp(c, SP_ZERO), c->stream, c->n_sm);
        launch_step_end(c->P, c->stream, 0, rebuild ? 1 : 0, 1, 0, 0, 0, 0);
        cudaEventRecord(e0, c->stream);
        launch_rebuild(c->P, c->stream, c->n_sm);
        launch_list_build(c->P, c->stream, c->max_lig_cl);
        cudaEventRecord(e1, c->stream);
        launch_prune(c->P, c->stream, c->n_sm);
        cudaEventRecord(e2, c->stream);
        float a = 0.f, b = 0.f, e = 0.f;
        cudaEventSynchronize(e2);
        cudaEventElapsedTime(&a, e0, e1);
        cudaEventElapsedTime(&b, e1, e2);
        cudaEventRecord(e0, c->stream);
        launch_env_forces(c->P, c->stream, false, c->prm.precision, c->env_grid,
                          c->tune.block_threads);
        cudaEventRecord(e1, c->stream);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&e, e0, e1);
        build_ms = a;
        prune_ms = b;
        env_ms = e;
        return check_device(c) == ABFE_OK;
    };
    abfe_tuning best = base;
    double best_cost = 1e300;
    for (double sk : cand) {
        if (sk > c->skin_cap + 1e-12 || st) continue;
        abfe_tuning t = base;
        t.graph_steps = 0;
        t.skin = sk;
        t.prune_skin = std::min(sk, pcand[0]);
        if (abfe_set_tuning(c, &t) != ABFE_OK) continue;
        float bm = 0.f, pm = 0.f, em = 0.f;
        if (!timed(true, bm, pm, em) || !timed(true, bm, pm, em)) continue;   // warm, then timed
        const double n_b = std::max(1.0, steps_to(0.5 * sk));
        for (double ps : pcand) {
            if (ps > sk + 1e-12 || ps > PRUNE_SKIN_MAX + 1e-12) continue;
            t.prune_skin = ps;
            if (abfe_set_tuning(c, &t) != ABFE_OK) continue;
            float b2 = 0.f;
            if (!timed(false, b2, pm, em)) continue;
            // per rebuild cycle: one build, a prune with it and one every n_p steps
            const double n_p = std::max(1.0, steps_to(0.5 * ps));
            const double prunes = std::ceil(n_b / n_p);
            const double cost = em + (bm + prunes * pm) / n_b;
            if (cost < best_cost) {
                best_cost = cost;
                best = base;
                best.skin = sk;
                best.prune_skin = ps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    c->prof_max = saved_prof;
    c->ex_every = saved_ex;
    c->P.ex_every = saved_ex;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (st) return st;
    st = abfe_set_tuning(c, &best);
    if (st) return st;
    return restore_state(c, saved);
}

// checkpoint (version 3): magic, version, R, total atoms, step, maxdisp2 bits,
// exchange attempts, positions, velocities, positions at the last prune and at
// the last outer list build (all [total][3] doubles), schedule and state of every
// replica. Versions 1 and 2 (no build positions) are read as well.
abfe_status abfe_save_checkpoint(abfe_ctx* c, const char* path) {
    if (!c || !path) return ABFE_ERR_INVALID_ARG;
    const size_t n3 = 3 * (size_t)c->total_atoms;
    abfe_status st = sync_states(c);
    if (st) return st;
    HostState h;
    st = save_state(c, h);
    if (st) return st;
    const std::vector<double>&x = h.x, &v = h.v, &xp = h.xp, &xb = h.xb;
    std::ofstream o(path, std::ios::binary);
    if (!o) return set_error(c, ABFE_ERR_INVALID_ARG, "cannot open checkpoint for writing");
    const uint64_t magic = 0x31504B4345464241ull;  // "ABFECKP1"
    const int64_t hdr[7] = {3, c->R, c->total_atoms, (int64_t)h.step, (int64_t)h.maxdisp2,
                            (int64_t)h.ex_attempt, (int64_t)h.ex_accepted};
    o.write((const char*)&magic, 8);
    o.write((const char*)hdr, sizeof hdr);
    o.write((const char*)x.data(), sizeof(double) * n3);
    o.write((const char*)v.data(), sizeof(double) * n3);
    o.write((const char*)xp.data(), sizeof(double) * n3);
    o.write((const char*)xb.data(), sizeof(double) * n3);
    std::vector<int32_t> ss(2 * c->R, 0);
    for (int r = 0; r < c->R && c->states_set; ++r) {
        ss[2 * r] = c->sched_of_rep[r];
        ss[2 * r + 1] = c->state_of_rep[r];
    }
    o.write((const char*)ss.data(), sizeof(int32_t) * ss.size());
    if (!o) return set_error(c, ABFE_ERR_INVALID_ARG, "checkpoint write failed");
    return ABFE_OK;
}

abfe_status abfe_load_checkpoint(abfe_ctx* c, const char* path) {
    if (!c || !path) return ABFE_ERR_INVALID_ARG;
    std::ifstream in(path, std::ios::binary);
    if (!in) return set_error(c, ABFE_ERR_INVALID_ARG, "cannot open checkpoint");
    uint64_t magic = 0;
    int64_t hdr[7] = {0, 0, 0, 0, 0, 0, 0};
    in.read((char*)&magic, 8);
    in.read((char*)hdr, 5 * sizeof(int64_t));
    if (in && hdr[0] >= 2) in.read((char*)(hdr + 5), sizeof(int64_t));
    if (in && hdr[0] >= 3) in.read((char*)(hdr + 6), sizeof(int64_t));
    if (!in || magic != 0x31504B4345464241ull || hdr[0] < 1 || hdr[0] > 3 || hdr[1] != c->R ||
        hdr[2] != c->total_atoms)
        return set_error(c, ABFE_ERR_INVALID_ARG, "checkpoint does not match this context");
    const size_t n3 = 3 * (size_t)c->total_atoms;
    std::vector<double> x(n3), v(n3), xp(n3), xb;
    in.read((char*)x.data(), sizeof(double) * n3);
    in.read((char*)v.data(), sizeof(double) * n3);
    in.read((char*)xp.data(), sizeof(double) * n3);
    if (hdr[0] >= 3) {
        xb.resize(n3);
        in.read((char*)xb.data(), sizeof(double) * n3);
    } else {
        xb = xp;   // earlier versions: the list was built and pruned at the same positions
    }
    std::vector<int32_t> ss(2 * c->R);
    in.read((char*)ss.data(), sizeof(int32_t) * ss.size());
    if (!in) return set_error(c, ABFE_ERR_INVALID_ARG, "truncated checkpoint");
    HostState h;
    h.x = std::move(x);
    h.v = std::move(v);
    h.xp = std::move(xp);
    h.xb = std::move(xb);
    h.step = (unsigned long long)hdr[3];
    h.maxdisp2 = (unsigned int)hdr[4];
    h.steps_done = c->steps_done;
    h.ex_attempt = (unsigned long long)hdr[5];
    h.ex_accepted = (long long)hdr[6];
    abfe_status st = restore_state(c, h);
    if (st) return st;
    std::vector<int32_t> sch(c->R), sta(c->R);
    bool have = true;
    for (int r = 0; r < c->R; ++r) {
        sch[r] = ss[2 * r];
        sta[r] = ss[2 * r + 1];
        if (c->sched[sch[r]].K == 0) have = false;
    }
    if (have) {
        st = abfe_set_replica_states(c, sch.data(), sta.data());
        if (st) return st;
    }
    c->f_valid = false;
    return ABFE_OK;
}

}  // extern "C"
