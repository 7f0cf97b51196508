"""ctypes binding of libabfe.so (include/abfe.h). Argument marshalling only:
every step of the computation runs in the library's CUDA kernels. There is no
fallback: if the library is missing the import of `lib()` raises."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libabfe.so")

N_ENERGY = 11
ENERGY_NAMES = ("env_lj", "env_coul", "ligenv_lj", "liglig_lj", "ligenv_coul", "liglig_coul",
                "bond", "restraint", "recip", "torsion", "total")
N_DUDL = 3
DUDL_NAMES = ("restraint", "coul", "vdw")

STATUS = {0: "ok", 1: "invalid argument", 2: "cutoff too large", 3: "list overflow",
          4: "non-finite", 5: "CUDA error", 6: "timeout", 7: "not implemented",
          8: "wrong call order", 9: "out of memory"}


class AbfeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"abfe error {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class SystemDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("box", C.c_double * 3),
                ("pos", C.c_void_p), ("vel", C.c_void_p), ("mass", C.c_void_p),
                ("charge", C.c_void_p), ("sigma", C.c_void_p), ("epsilon", C.c_void_p),
                ("is_ligand", C.c_void_p), ("n_excl", C.c_int32), ("excl", C.c_void_p),
                ("n_bonds", C.c_int32), ("bond_idx", C.c_void_p), ("bond_r0", C.c_void_p),
                ("bond_k", C.c_void_p), ("has_boresch", C.c_int32), ("anchors", C.c_int32 * 6),
                ("b_r0", C.c_double), ("b_theta0", C.c_double * 2), ("b_phi0", C.c_double * 3),
                ("b_kr", C.c_double), ("b_ktheta", C.c_double), ("b_kphi", C.c_double),
                ("n_torsions", C.c_int32), ("torsion_idx", C.c_void_p), ("torsion_k", C.c_void_p),
                ("torsion_n", C.c_void_p), ("torsion_phi0", C.c_void_p),
                ("n_alch_waters", C.c_int32), ("alch_water_idx", C.c_void_p),
                ("alch_water_dq", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("cutoff", C.c_double), ("ewald_beta", C.c_double), ("sc_alpha", C.c_double),
                ("sc_p", C.c_double), ("coulomb_k", C.c_double), ("kT", C.c_double),
                ("skin", C.c_double), ("ligand_mode", C.c_int32), ("precision", C.c_int32),
                ("pme_spacing", C.c_double), ("pme_order", C.c_int32), ("pme_reserved", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("group", C.c_int32), ("max_entries", C.c_int32),
                ("block_threads", C.c_int32), ("graph_steps", C.c_int32), ("skin", C.c_double),
                ("prune_skin", C.c_double), ("reserved0", C.c_int32), ("reserved1", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("env_ms", C.c_double), ("env_launches", C.c_int64), ("lig_ms", C.c_double),
                ("lig_launches", C.c_int64), ("integrate_ms", C.c_double),
                ("integrate_launches", C.c_int64), ("build_ms", C.c_double),
                ("build_launches", C.c_int64), ("prune_ms", C.c_double),
                ("prune_launches", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("n_items_env", C.c_int64), ("n_items_lig", C.c_int64),
                ("n_entries", C.c_int64), ("n_xentries", C.c_int64), ("n_rebuilds", C.c_int64),
                ("steps_done", C.c_int64), ("slots", C.c_int64), ("clusters", C.c_int64),
                ("device_bytes", C.c_int64), ("env_lane_groups", C.c_int64),
                ("n_prunes", C.c_int64), ("n_rows", C.c_int64), ("n_xrows", C.c_int64),
                ("n_exchange_attempts", C.c_int64), ("n_exchange_accepted", C.c_int64),
                ("n_window_rebuilds", C.c_int64), ("n_window_prunes", C.c_int64)]


NOALLOC_MAX_K = 128
NOALLOC_MAX_EXCL = 16


class NoallocFrame(C.Structure):
    """abfe_noalloc_frame: inputs of abfe_ukn_frame_noalloc (device pointers + host values)."""
    _fields_ = [("n_atoms", C.c_int32), ("box", C.c_double * 3), ("pos", C.c_void_p),
                ("charge", C.c_void_p), ("sigma", C.c_void_p), ("epsilon", C.c_void_p),
                ("is_ligand", C.c_void_p), ("n_lig", C.c_int32), ("lig_idx", C.c_void_p),
                ("lig_excl", C.c_void_p), ("K", C.c_int32),
                ("lam_r", C.c_double * NOALLOC_MAX_K), ("lam_q", C.c_double * NOALLOC_MAX_K),
                ("lam_v", C.c_double * NOALLOC_MAX_K), ("cutoff", C.c_double),
                ("ewald_beta", C.c_double), ("sc_alpha", C.c_double), ("sc_p", C.c_double),
                ("coulomb_k", C.c_double), ("ligand_mode", C.c_int32), ("has_boresch", C.c_int32),
                ("anchors", C.c_int32 * 6), ("b_r0", C.c_double), ("b_theta0", C.c_double * 2),
                ("b_phi0", C.c_double * 3), ("b_kr", C.c_double), ("b_ktheta", C.c_double),
                ("b_kphi", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)

# (name, argtypes, restype)
_SIGS = [
    ("abfe_set_allocator", [ALLOC_FN, FREE_FN, C.c_void_p], None),
    ("abfe_create", [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                     C.POINTER(C.c_void_p)], C.c_int),
    ("abfe_set_lambda_schedule", [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                  C.c_void_p], C.c_int),
    ("abfe_set_replica_states", [C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_build_neighbor_list", [C.c_void_p], C.c_int),
    ("abfe_compute", [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_compute_device", [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_step", [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.c_uint64], C.c_int),
    ("abfe_eval_ukn", [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    ("abfe_get_positions", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_set_positions", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_get_velocities", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_set_velocities", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_count_pairs", [C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_set_tuning", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_get_tuning", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_autotune", [C.c_void_p, C.c_char_p, C.c_int32], C.c_int),
    ("abfe_get_stats", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_autotune_cadence", [C.c_void_p, C.c_double, C.c_double, C.c_uint64, C.c_int32], C.c_int),
    ("abfe_set_profiling", [C.c_void_p, C.c_int32], C.c_int),
    ("abfe_get_profile", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_save_checkpoint", [C.c_void_p, C.c_char_p], C.c_int),
    ("abfe_load_checkpoint", [C.c_void_p, C.c_char_p], C.c_int),
    ("abfe_num_replicas", [C.c_void_p], C.c_int32),
    ("abfe_total_atoms", [C.c_void_p], C.c_int64),
    ("abfe_atom_offset", [C.c_void_p, C.c_int32], C.c_int64),
    ("abfe_last_error", [C.c_void_p], C.c_char_p),
    ("abfe_status_string", [C.c_int], C.c_char_p),
    ("abfe_destroy", [C.c_void_p], None),
    ("abfe_ukn_frame_noalloc", [C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_boresch_correction", [C.c_double, C.c_double, C.c_void_p, C.c_double, C.c_double,
                                 C.c_double, C.c_void_p], C.c_int),
    ("abfe_replica_exchange", [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int32, C.c_void_p,
                               C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_get_replica_states", [C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_set_exchange", [C.c_void_p, C.c_int32, C.c_uint64], C.c_int),
    ("abfe_mbar", [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int32,
                   C.c_void_p, C.c_void_p], C.c_int),
    ("abfe_mbar_device", [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int32,
                          C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
]

_lib = None


def lib():
    """Load libabfe.so (built by paper_2603_22274_gb300.build). Raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_2603_22274_gb300.build`"
                               " (or __graft_entry__.build()); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, args, res in _SIGS:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols() -> Sequence[str]:
    return [s[0] for s in _SIGS]


_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          int(stream or 0)))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    lib().abfe_set_allocator(_torch_hooks[0], _torch_hooks[1], None)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def boresch_correction(kT, r0, theta0, k_r, k_theta, k_phi):
    """Free energy (kJ/mol) of imposing the Boresch restraint on the decoupled
    ligand at 1 mol/L (abfe_boresch_correction)."""
    th = np.ascontiguousarray(theta0, dtype=np.float64)
    out = C.c_double(0.0)
    st = lib().abfe_boresch_correction(float(kT), float(r0), _ptr(th), float(k_r), float(k_theta),
                                       float(k_phi), C.byref(out))
    if st != 0:
        raise AbfeError(st, lib().abfe_last_error(None).decode())
    return out.value


def mbar(u_kn, N_k, tol=1e-12, max_iter=100000, stream=None):
    """MBAR free energies (f_0 = 0, kT units) and the iteration count, through
    abfe_mbar (host array) or abfe_mbar_device (a CUDA torch tensor, FP64,
    contiguous [K][N]); all arithmetic runs in the library's kernels."""
    n_k = np.ascontiguousarray(N_k, dtype=np.int32)
    K = int(n_k.shape[0])
    f = np.zeros(K)
    it = C.c_int32(0)
    if hasattr(u_kn, "data_ptr"):
        import torch
        assert u_kn.dtype == torch.float64 and u_kn.is_cuda and u_kn.is_contiguous()
        assert u_kn.dim() == 2 and u_kn.shape[0] == K
        N = int(u_kn.shape[1])
        if stream is None:
            stream = torch.cuda.current_stream()
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        st = lib().abfe_mbar_device(C.c_void_p(u_kn.data_ptr()), _ptr(n_k), K, N, float(tol),
                                    int(max_iter), _ptr(f), C.byref(it), C.c_void_p(sp))
    else:
        u = np.ascontiguousarray(u_kn, dtype=np.float64)
        assert u.ndim == 2 and u.shape[0] == K
        N = int(u.shape[1])
        st = lib().abfe_mbar(_ptr(u), _ptr(n_k), K, N, float(tol), int(max_iter), _ptr(f),
                             C.byref(it))
    if st != 0:
        raise AbfeError(st, lib().abfe_last_error(None).decode())
    return f, it.value


class Engine:
    """One context: several systems, each simulated by one or more replicas.

    systems: objects with n, box, pos, vel, mass, charge, sigma, epsilon,
    is_ligand, excl, bonds, bond_r0, bond_k and boresch (None or an object with
    anchors, r0, theta0, phi0, k_r, k_theta, k_phi).
    params: dict with cutoff, ewald_beta, sc_alpha, sc_p, coulomb_k, kT, skin,
    ligand_mode and optionally precision.
    stream: a torch.cuda.Stream, a raw cudaStream_t (int) or None (the library
    then creates its own stream).
    """

    def __init__(self, systems, system_of_replica, params, stream=None, torch_alloc=True,
                 precision=None):
        L = lib()
        if torch_alloc:
            use_torch_allocator()
        self._keep = []
        descs = (SystemDesc * len(systems))()
        for k, s in enumerate(systems):
            d = descs[k]
            arrs = dict(pos=_f64(s.pos, (-1, 3)), vel=_f64(s.vel, (-1, 3)), mass=_f64(s.mass),
                        charge=_f64(s.charge), sigma=_f64(s.sigma), epsilon=_f64(s.epsilon),
                        lig=np.ascontiguousarray(s.is_ligand, dtype=np.uint8),
                        excl=np.ascontiguousarray(s.excl, dtype=np.int32).reshape(-1, 2),
                        bonds=np.ascontiguousarray(s.bonds, dtype=np.int32).reshape(-1, 2),
                        r0=_f64(s.bond_r0), kb=_f64(s.bond_k),
                        tidx=np.ascontiguousarray(getattr(s, "torsions", np.zeros((0, 4))),
                                                  dtype=np.int32).reshape(-1, 4),
                        tk=_f64(getattr(s, "torsion_k", np.zeros(0))),
                        tn=np.ascontiguousarray(getattr(s, "torsion_n", np.zeros(0)), dtype=np.int32),
                        tp=_f64(getattr(s, "torsion_phi0", np.zeros(0))),
                        aw=np.ascontiguousarray(getattr(s, "alch_water", np.zeros(0)), dtype=np.int32),
                        awq=_f64(getattr(s, "alch_water_dq", np.zeros(0))))
            self._keep.append(arrs)
            d.n_atoms = int(arrs["pos"].shape[0])
            for i in range(3):
                d.box[i] = float(s.box[i])
            d.pos, d.vel, d.mass = _ptr(arrs["pos"]), _ptr(arrs["vel"]), _ptr(arrs["mass"])
            d.charge, d.sigma, d.epsilon = _ptr(arrs["charge"]), _ptr(arrs["sigma"]), _ptr(arrs["epsilon"])
            d.is_ligand = _ptr(arrs["lig"])
            d.n_excl, d.excl = len(arrs["excl"]), _ptr(arrs["excl"])
            d.n_bonds, d.bond_idx = len(arrs["bonds"]), _ptr(arrs["bonds"])
            d.bond_r0, d.bond_k = _ptr(arrs["r0"]), _ptr(arrs["kb"])
            d.n_torsions = len(arrs["tidx"])
            d.torsion_idx, d.torsion_k = _ptr(arrs["tidx"]), _ptr(arrs["tk"])
            d.torsion_n, d.torsion_phi0 = _ptr(arrs["tn"]), _ptr(arrs["tp"])
            d.n_alch_waters = len(arrs["aw"])
            d.alch_water_idx, d.alch_water_dq = _ptr(arrs["aw"]), _ptr(arrs["awq"])
            b = getattr(s, "boresch", None)
            d.has_boresch = 1 if b is not None else 0
            if b is not None:
                for i in range(6):
                    d.anchors[i] = int(b.anchors[i])
                d.b_r0 = float(b.r0)
                d.b_theta0[0], d.b_theta0[1] = float(b.theta0[0]), float(b.theta0[1])
                for i in range(3):
                    d.b_phi0[i] = float(b.phi0[i])
                d.b_kr, d.b_ktheta, d.b_kphi = float(b.k_r), float(b.k_theta), float(b.k_phi)
        sor = np.ascontiguousarray(system_of_replica, dtype=np.int32)
        prec = int(params.get("precision", 0) if precision is None else precision)
        self.params = dict(params)
        p = Params(params["cutoff"], params["ewald_beta"], params["sc_alpha"], params["sc_p"],
                   params["coulomb_k"], params["kT"], params.get("skin", 0.1),
                   int(params.get("ligand_mode", 0)), prec,
                   float(params.get("pme_spacing", 0.0)), int(params.get("pme_order", 0)), 0)
        if stream is None:
            h = None
        elif isinstance(stream, int):
            h = stream
        else:
            h = int(stream.cuda_stream)
        self._stream = stream
        out = C.c_void_p()
        st = L.abfe_create(C.byref(descs), len(systems), _ptr(sor), len(sor), C.byref(p), h,
                           C.byref(out))
        if st != 0:
            raise AbfeError(st, L.abfe_last_error(None).decode())
        self._ctx = out
        self.R = int(L.abfe_num_replicas(out))
        self.total_atoms = int(L.abfe_total_atoms(out))
        self.offsets = np.array([L.abfe_atom_offset(out, r) for r in range(self.R)] +
                                [self.total_atoms], dtype=np.int64)
        self.K = {}

    # ------------------------------------------------------------------ plumbing
    def _ck(self, st):
        if st != 0:
            raise AbfeError(st, lib().abfe_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None):
            lib().abfe_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ states
    def set_schedule(self, sid, lam_r, lam_q, lam_v):
        lr, lq, lv = _f64(lam_r), _f64(lam_q), _f64(lam_v)
        self._ck(lib().abfe_set_lambda_schedule(self._ctx, int(sid), len(lr), _ptr(lr), _ptr(lq), _ptr(lv)))
        self.K[int(sid)] = len(lr)

    def set_states(self, schedule_of_replica, state_of_replica):
        a = np.ascontiguousarray(schedule_of_replica, dtype=np.int32)
        b = np.ascontiguousarray(state_of_replica, dtype=np.int32)
        self._ck(lib().abfe_set_replica_states(self._ctx, _ptr(a), _ptr(b)))
        self._sched_of = a

    def build_list(self):
        self._ck(lib().abfe_build_neighbor_list(self._ctx))

    # ------------------------------------------------------------------ evaluation
    def compute(self, forces=True):
        F = np.zeros((self.total_atoms, 3)) if forces else None
        E = np.zeros((self.R, N_ENERGY))
        D = np.zeros((self.R, N_DUDL))
        self._ck(lib().abfe_compute(self._ctx, _ptr(F), _ptr(E), _ptr(D)))
        return F, E, D

    def compute_device(self, d_forces=None, d_energy=None, d_dudl=None):
        """Device-output variant; arguments are CUDA tensors (or raw pointers)."""
        def p(t):
            if t is None:
                return None
            return t if isinstance(t, int) else int(t.data_ptr())
        self._ck(lib().abfe_compute_device(self._ctx, p(d_forces), p(d_energy), p(d_dudl)))

    def step(self, n, dt=0.001, gamma=1.0, seed=1):
        self._ck(lib().abfe_step(self._ctx, int(n), float(dt), float(gamma), int(seed)))

    def eval_ukn(self, ld=None):
        if ld is None:
            ld = max(self.K.values())
        U = np.zeros((self.R, ld))
        dU = np.zeros((self.R, ld))
        D = np.zeros((self.R, N_DUDL))
        self._ck(lib().abfe_eval_ukn(self._ctx, _ptr(U), _ptr(dU), int(ld), _ptr(D)))
        return U, dU, D

    def replica_exchange(self, seed, ukn=None, ld=None, return_ukn=False):
        """One neighbour-exchange attempt on the device (abfe_replica_exchange).
        ukn: host [R][ld] reduced potentials to decide with, or None to evaluate
        them on the device. Returns (states after, accepted swaps[, u_kn used])."""
        if ld is None:
            ld = max(self.K.values()) if ukn is None else int(np.asarray(ukn).shape[1])
        st = np.zeros(self.R, np.int32)
        acc = C.c_int32(0)
        u_in = None if ukn is None else _f64(ukn, (self.R, ld))
        u_out = np.zeros((self.R, ld)) if (return_ukn and ukn is None) else None
        self._ck(lib().abfe_replica_exchange(self._ctx, int(seed), _ptr(u_in), int(ld), _ptr(u_out),
                                             _ptr(st), C.byref(acc)))
        return (st, acc.value, u_out) if return_ukn else (st, acc.value)

    def set_exchange(self, every_steps, seed=1):
        """Replica exchange inside abfe_step every `every_steps` steps (0 = off)."""
        self._ck(lib().abfe_set_exchange(self._ctx, int(every_steps), int(seed)))

    def replica_states(self):
        st = np.zeros(self.R, np.int32)
        self._ck(lib().abfe_get_replica_states(self._ctx, _ptr(st)))
        return st

    def positions(self):
        x = np.zeros((self.total_atoms, 3))
        self._ck(lib().abfe_get_positions(self._ctx, _ptr(x)))
        return x

    def set_positions(self, x):
        x = _f64(x, (-1, 3))
        self._ck(lib().abfe_set_positions(self._ctx, _ptr(x)))

    def velocities(self):
        v = np.zeros((self.total_atoms, 3))
        self._ck(lib().abfe_get_velocities(self._ctx, _ptr(v)))
        return v

    def set_velocities(self, v):
        v = _f64(v, (-1, 3))
        self._ck(lib().abfe_set_velocities(self._ctx, _ptr(v)))

    def count_pairs(self, per_atom=False):
        c = np.zeros((self.R, 2), np.int64)
        a = np.zeros(self.total_atoms, np.int32) if per_atom else None
        self._ck(lib().abfe_count_pairs(self._ctx, _ptr(c), _ptr(a)))
        return (c, a) if per_atom else c

    # ------------------------------------------------------------------ tuning / stats
    def tuning(self):
        t = Tuning()
        self._ck(lib().abfe_get_tuning(self._ctx, C.byref(t)))
        return dict(group=t.group, max_entries=t.max_entries, block_threads=t.block_threads,
                    graph_steps=t.graph_steps, skin=t.skin, prune_skin=t.prune_skin)

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        if "skin" in kw and "prune_skin" not in kw:
            cur["prune_skin"] = min(cur["prune_skin"], cur["skin"])
        t = Tuning(cur["group"], cur["max_entries"], cur["block_threads"], cur["graph_steps"],
                   cur["skin"], cur["prune_skin"], 0, 0)
        self._ck(lib().abfe_set_tuning(self._ctx, C.byref(t)))

    def autotune_cadence(self, dt=0.001, gamma=1.0, seed=1, n_steps=48):
        self._ck(lib().abfe_autotune_cadence(self._ctx, float(dt), float(gamma), int(seed),
                                             int(n_steps)))
        return self.tuning()

    def autotune(self, cache_path=None, reps=3):
        cp = cache_path.encode() if cache_path else None
        self._ck(lib().abfe_autotune(self._ctx, cp, int(reps)))
        return self.tuning()

    def stats(self):
        s = Stats()
        self._ck(lib().abfe_get_stats(self._ctx, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def set_profiling(self, max_launches):
        self._ck(lib().abfe_set_profiling(self._ctx, int(max_launches)))

    def profile(self):
        p = Profile()
        self._ck(lib().abfe_get_profile(self._ctx, C.byref(p)))
        return {k: getattr(p, k) for k, _ in Profile._fields_}

    def save_checkpoint(self, path):
        self._ck(lib().abfe_save_checkpoint(self._ctx, path.encode()))

    def load_checkpoint(self, path):
        self._ck(lib().abfe_load_checkpoint(self._ctx, path.encode()))


def engine_for_workload(w, stream=None, precision=None, torch_alloc=True) -> Engine:
    """Create an Engine for an abfe_synth.Workload-like object and set its states."""
    e = Engine(w.systems, w.system_of_replica, w.params, stream=stream, precision=precision,
               torch_alloc=torch_alloc)
    for sid, sch in enumerate(w.schedules):
        e.set_schedule(sid, sch.lam_r, sch.lam_q, sch.lam_v)
    e.set_states(w.schedule_of_replica, w.state_of_replica)
    return e
