"""ctypes binding of libphoebe_gpu.so (argument marshalling only).

Every step of the computation runs in the CUDA library; this module converts
numpy arrays / torch tensors to pointers and sizes and raises on a non-zero
status.  There is no CPU fallback: if the shared library is missing or fails
to load, importing the package raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PHOEBE_GPU_LIB may name another build of the library (same ABI)
LIB_PATH = os.environ.get("PHOEBE_GPU_LIB") or os.path.join(_HERE, "libphoebe_gpu.so")

STATUS = {
    0: "OK", -1: "ERR_ARG", -2: "ERR_ORDER", -3: "ERR_SHAPE", -4: "ERR_GRID", -5: "ERR_NOMEM",
    -6: "ERR_CUDA", -7: "ERR_TIMEOUT", -8: "ERR_NOTCONVERGED", -9: "ERR_UNSUPPORTED",
}
PREC_FP64, PREC_SPLIT_BF16, PREC_SPLIT_TF32, PREC_BF16, PREC_TF32, PREC_SPLIT_FP16, PREC_BF16X3 = 0, 1, 2, 3, 4, 5, 6
PREC_FP32_DFT = 7
PREC_FP64_DFT = 8
SAMPLER_FULL, SAMPLER_LEARNED, SAMPLER_UNIFORM, SAMPLER_SHELL = 0, 1, 2, 3
MLP_NPARAM = 34177

# symbols declared in include/phoebe_gpu.h
EXPORTED = (
    "phoebe_gpu_create", "phoebe_gpu_destroy", "phoebe_gpu_last_error",
    "phoebe_gpu_set_hamiltonian", "phoebe_gpu_set_force_constants", "phoebe_gpu_set_elph_wannier",
    "phoebe_gpu_interpolate_couplings", "phoebe_gpu_rta_params_default",
    "phoebe_gpu_linewidths_rta", "phoebe_gpu_linewidths_rta_dev",
    "phoebe_gpu_set_profiling", "phoebe_gpu_get_stats", "phoebe_gpu_set_memory_cap",
    "phoebe_gpu_constants", "phoebe_gpu_version", "phoebe_gpu_bands_noalloc",
    "phoebe_gpu_sampler_init", "phoebe_gpu_sampler_load", "phoebe_gpu_sampler_save",
    "phoebe_gpu_train_opts_default", "phoebe_gpu_sampler_train", "phoebe_gpu_q_contributions",
    "phoebe_gpu_mlp_loss_grad", "phoebe_gpu_is_uniforms", "phoebe_gpu_mlp_scores",
    "phoebe_gpu_batch_opts_default", "phoebe_gpu_linewidths_rta_batch", "phoebe_gpu_transport_rta",
    "phoebe_gpu_selftest_wait", "phoebe_gpu_selftest_fp32_rate", "phoebe_gpu_phonon_rates_elph", "phoebe_gpu_set_lattice",
    "phoebe_gpu_set_polar", "phoebe_gpu_set_force_constants3", "phoebe_gpu_three_phonon_rates",
)


class PhoebeGPUError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class RTAParams(C.Structure):
    _fields_ = [
        ("nk", C.c_int * 3), ("nq", C.c_int * 3),
        ("T_K", C.c_double), ("mu_eV", C.c_double), ("sigma_eV", C.c_double), ("window_eV", C.c_double),
        ("delta_cut_sigmas", C.c_double), ("omega_cut_eV", C.c_double), ("degen_tol_eV", C.c_double),
        ("precision", C.c_int),
        ("n_k_subset", C.c_int), ("k_subset", C.POINTER(C.c_int32)),
        ("max_batch_states", C.c_int),
        ("sampler", C.c_int),
        ("sample_fraction", C.c_double), ("mix_alpha", C.c_double), ("seed", C.c_uint64),
        ("sampler_fp32_network", C.c_int), ("smearing", C.c_int),
        ("population_delta", C.c_double), ("sigma_min_eV", C.c_double),
        ("window_final", C.c_int), ("reserved1", C.c_int),
    ]


class TrainOpts(C.Structure):
    _fields_ = [
        ("epochs", C.c_int), ("states_per_step", C.c_int),
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
        ("seed", C.c_uint64),
        ("reserved", C.c_int * 4),
    ]


class BatchItem(C.Structure):
    _fields_ = [
        ("ctx", C.c_void_p), ("params", C.c_void_p), ("n_states", C.c_int),
        ("k_index", C.c_void_p), ("band", C.c_void_p), ("gamma_eV", C.c_void_p),
        ("tile_n", C.c_int), ("tile_kb", C.c_int),
    ]


class BatchOpts(C.Structure):
    _fields_ = [
        ("autotune", C.c_int), ("n_streams", C.c_int), ("g_chunk_bytes", C.c_int64),
        ("plan_ms", C.c_double), ("graph_ms", C.c_double), ("finish_ms", C.c_double),
        ("graph_nodes", C.c_int64), ("recorded_launches", C.c_int64),
        ("plan_threads", C.c_int), ("graph_reused", C.c_int), ("reserved", C.c_int * 2),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("n_states", C.c_int64), ("n_k", C.c_int64), ("n_q", C.c_int64),
        ("pairs_dense", C.c_int64), ("pairs_executed", C.c_int64),
        ("couplings_dense", C.c_int64), ("couplings_executed", C.c_int64),
        ("kernel_launches", C.c_int64), ("stage2_launches", C.c_int64),
        ("stage2_flops", C.c_double), ("stage2_ms", C.c_double),
        ("bands_ms", C.c_double), ("phonons_ms", C.c_double), ("window_ms", C.c_double),
        ("stage1_ms", C.c_double), ("rotate_ms", C.c_double), ("delta_ms", C.c_double),
        ("total_ms", C.c_double), ("sampler_ms", C.c_double),
    ]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2111_14999_b300.build`")
    lib = C.CDLL(LIB_PATH)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "phoebe_gpu_create": (I, [C.POINTER(P), I, P]),
        "phoebe_gpu_destroy": (I, [P]),
        "phoebe_gpu_last_error": (C.c_char_p, [P]),
        "phoebe_gpu_set_hamiltonian": (I, [P, I, I, P, P, P]),
        "phoebe_gpu_set_force_constants": (I, [P, I, P, I, P, P, P]),
        "phoebe_gpu_set_elph_wannier": (I, [P, I, P, P, I, P, P, P]),
        "phoebe_gpu_interpolate_couplings": (I, [P, I, P, P, I, P, P, P, P]),
        "phoebe_gpu_rta_params_default": (None, [C.POINTER(RTAParams)]),
        "phoebe_gpu_linewidths_rta": (I, [P, C.POINTER(RTAParams), C.POINTER(I), P, P, P]),
        "phoebe_gpu_linewidths_rta_dev": (I, [P, C.POINTER(RTAParams), C.POINTER(I), P, P, P]),
        "phoebe_gpu_set_profiling": (I, [P, I]),
        "phoebe_gpu_get_stats": (I, [P, C.POINTER(Stats)]),
        "phoebe_gpu_set_memory_cap": (I, [P, I64]),
        "phoebe_gpu_constants": (None, [C.POINTER(D)]),
        "phoebe_gpu_version": (C.c_char_p, []),
        "phoebe_gpu_bands_noalloc": (I, [I, I, P, P, P, I, P, P, P, P]),
        "phoebe_gpu_sampler_init": (I, [P, C.c_uint64]),
        "phoebe_gpu_sampler_load": (I, [P, P, I64]),
        "phoebe_gpu_sampler_save": (I, [P, P, I64]),
        "phoebe_gpu_train_opts_default": (None, [C.POINTER(TrainOpts)]),
        "phoebe_gpu_sampler_train": (I, [P, C.POINTER(RTAParams), C.POINTER(TrainOpts), P]),
        "phoebe_gpu_q_contributions": (I, [P, C.POINTER(RTAParams), C.POINTER(I), P, P, P, P, P]),
        "phoebe_gpu_mlp_loss_grad": (I, [P, I64, P, I, P, P, P, P, P, P]),
        "phoebe_gpu_is_uniforms": (I, [P, C.c_uint64, C.c_int32, I64, P]),
        "phoebe_gpu_mlp_scores": (I, [P, I, P, P, I, P]),
        "phoebe_gpu_batch_opts_default": (None, [C.POINTER(BatchOpts)]),
        "phoebe_gpu_linewidths_rta_batch": (I, [C.POINTER(BatchItem), I, C.POINTER(BatchOpts)]),
        "phoebe_gpu_transport_rta": (I, [P, C.POINTER(RTAParams), P, P, P, P]),
        "phoebe_gpu_phonon_rates_elph": (I, [P, C.POINTER(RTAParams), C.c_int64, P]),
        "phoebe_gpu_set_lattice": (I, [P, P]),
        "phoebe_gpu_set_polar": (I, [P, P, P, C.c_double]),
        "phoebe_gpu_set_force_constants3": (I, [P, C.c_int, P, P, P, P]),
        "phoebe_gpu_three_phonon_rates": (I, [P, C.POINTER(RTAParams), C.c_int64, P]),
        "phoebe_gpu_selftest_wait": (I, [P, I, I64]),
        "phoebe_gpu_selftest_fp32_rate": (I, [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def constants() -> tuple:
    out = (C.c_double * 3)()
    lib.phoebe_gpu_constants(out)
    return tuple(out)


def version() -> str:
    return lib.phoebe_gpu_version().decode()


def _ptr(a) -> C.c_void_p | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):          # torch tensor
        return C.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return C.c_void_p(a)
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128_as_f64(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def make_params(p=None, **kw) -> RTAParams:
    """Build the C params struct from a workloads.RTAParams-like object and/or keywords."""
    s = RTAParams()
    lib.phoebe_gpu_rta_params_default(C.byref(s))
    src = dict(p.__dict__) if p is not None else {}
    src.update(kw)
    keep = []
    for key, val in src.items():
        if val is None:
            continue
        if key in ("nk", "nq"):
            getattr(s, key)[:] = [int(v) for v in val]
        elif key == "k_subset":
            arr = _i32(val)
            keep.append(arr)
            s.n_k_subset = len(arr)
            s.k_subset = arr.ctypes.data_as(C.POINTER(C.c_int32))
        elif key in ("T_K", "mu_eV", "sigma_eV", "window_eV", "delta_cut_sigmas", "omega_cut_eV", "degen_tol_eV"):
            setattr(s, key, float(val))
        elif key in ("precision", "max_batch_states", "sampler", "seed", "sampler_fp32_network", "smearing",
                     "window_final"):
            setattr(s, key, int(val))
        elif key in ("sample_fraction", "mix_alpha", "population_delta", "sigma_min_eV"):
            setattr(s, key, float(val))
    s._keep = keep  # keep the subset array alive with the struct
    return s


class PhoebeGPU:
    """One library context on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self._ctx = C.c_void_p()
        handle = None
        if stream is not None:
            handle = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = lib.phoebe_gpu_create(C.byref(self._ctx), int(device), handle)
        if st != 0:
            raise PhoebeGPUError(st, f"phoebe_gpu_create(device={device}) failed")

    # -------------------------------------------------------------- plumbing
    def _check(self, st: int):
        if st != 0:
            raise PhoebeGPUError(st, lib.phoebe_gpu_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            lib.phoebe_gpu_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -------------------------------------------------------------- inputs
    def set_hamiltonian(self, nw, R, w, H):
        R, H = _i32(R), _c128_as_f64(H)
        w = None if w is None else _f64(w)
        self._check(lib.phoebe_gpu_set_hamiltonian(self._ctx, int(nw), len(R), _ptr(R), _ptr(w), _ptr(H)))

    def set_force_constants(self, na, mass_amu, R, w, Phi):
        m, R, Phi = _f64(mass_amu), _i32(R), _f64(Phi)
        w = None if w is None else _f64(w)
        self._check(lib.phoebe_gpu_set_force_constants(self._ctx, int(na), _ptr(m), len(R), _ptr(R), _ptr(w),
                                                       _ptr(Phi)))

    def set_elph_wannier(self, Re, we, Rp, wp, g):
        Re, Rp = _i32(Re), _i32(Rp)
        we = None if we is None else _f64(we)
        wp = None if wp is None else _f64(wp)
        g = _c128_as_f64(g)
        self._check(lib.phoebe_gpu_set_elph_wannier(self._ctx, len(Re), _ptr(Re), _ptr(we), len(Rp), _ptr(Rp),
                                                    _ptr(wp), _ptr(g)))

    def set_material(self, mat):
        """All three set_* calls from an object with the workloads.Material fields."""
        self.set_hamiltonian(mat.nw, mat.R_H, mat.w_H, mat.H)
        self.set_force_constants(mat.na, mat.mass_amu, mat.R_fc, mat.w_fc, mat.Phi)
        self.set_elph_wannier(mat.Re, mat.we, mat.Rp, mat.wp, mat.g)
        if getattr(mat, "lattice", None) is not None:
            self.set_lattice(mat.lattice)
        self.nw, self.na = int(mat.nw), int(mat.na)

    def set_force_constants3(self, anh):
        """Third-order force constants from an object with the workloads.Anharmonic fields."""
        R, Rp = _i32(anh.R).reshape(-1, 3), _i32(anh.Rp).reshape(-1, 3)
        w = _f64(anh.w)
        phi = _f64(anh.Phi3)
        self._check(lib.phoebe_gpu_set_force_constants3(self._ctx, len(R), _ptr(R), _ptr(Rp), _ptr(w), _ptr(phi)))

    def three_phonon_rates(self, params, n_modes: int, **kw):
        """Three-phonon diagonal of the phonon scattering matrix A[q, nu] (eV) on the q grid."""
        s = params if isinstance(params, RTAParams) else make_params(params, **kw)
        nq = int(s.nq[0]) * int(s.nq[1]) * int(s.nq[2])
        out = np.empty((nq, int(n_modes)), dtype=np.float64)
        self._check(lib.phoebe_gpu_three_phonon_rates(self._ctx, C.byref(s), C.c_int64(out.size), _ptr(out)))
        return out

    def set_polar(self, Zstar=None, eps_inf=None, alpha: float = 1.0):
        """Born charges (na, 3, 3), eps_inf (3, 3) and the Gaussian filter alpha (1/A^2) of the polar
        long-range coupling; Zstar=None switches it off."""
        if Zstar is None:
            self._check(lib.phoebe_gpu_set_polar(self._ctx, None, None, C.c_double(0.0)))
            return
        zs = np.ascontiguousarray(Zstar, dtype=np.float64).reshape(-1)
        ep = np.ascontiguousarray(eps_inf, dtype=np.float64).reshape(9)
        self._check(lib.phoebe_gpu_set_polar(self._ctx, _ptr(zs), _ptr(ep), C.c_double(alpha)))

    def set_lattice(self, lattice):
        """Primitive lattice vectors (rows, Cartesian, Angstrom)."""
        lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
        self._check(lib.phoebe_gpu_set_lattice(self._ctx, _ptr(lat)))

    # -------------------------------------------------------------- compute
    def interpolate_couplings(self, k, q, precision: int = PREC_FP64, nw: int | None = None,
                              na: int | None = None):
        k, q = _f64(k).reshape(-1, 3), _f64(q).reshape(-1, 3)
        n = len(k)
        nw = nw or self.nw
        nm = 3 * (na or self.na)
        g2 = np.empty((n, nw, nw, nm))
        ek = np.empty((n, nw))
        ekq = np.empty((n, nw))
        om = np.empty((n, nm))
        self._check(lib.phoebe_gpu_interpolate_couplings(self._ctx, n, _ptr(k), _ptr(q), int(precision), _ptr(g2),
                                                         _ptr(ek), _ptr(ekq), _ptr(om)))
        return g2, ek, ekq, om

    def count_states(self, params) -> int:
        s = params if isinstance(params, RTAParams) else make_params(params)
        n = C.c_int(0)
        self._check(lib.phoebe_gpu_linewidths_rta(self._ctx, C.byref(s), C.byref(n), None, None, None))
        return n.value

    def linewidths_rta(self, params, capacity: int | None = None, **kw):
        """Host-buffer call: returns (k_index, band, gamma_eV) numpy arrays.  With `capacity`
        (an upper bound of the active-state count) the counting call is skipped."""
        s = params if isinstance(params, RTAParams) else make_params(params, **kw)
        n = self.count_states(s) if capacity is None else int(capacity)
        ki = np.empty(max(n, 1), dtype=np.int32)
        bd = np.empty(max(n, 1), dtype=np.int32)
        gm = np.empty(max(n, 1), dtype=np.float64)
        nn = C.c_int(max(n, 1))
        self._check(lib.phoebe_gpu_linewidths_rta(self._ctx, C.byref(s), C.byref(nn), _ptr(ki), _ptr(bd), _ptr(gm)))
        m = nn.value
        return ki[:m], bd[:m], gm[:m]

    def linewidths_rta_dev(self, params, k_index_dev, band_dev, gamma_dev, capacity: int) -> int:
        """Device-buffer call (torch tensors or raw device pointers); returns the state count."""
        s = params if isinstance(params, RTAParams) else make_params(params)
        nn = C.c_int(int(capacity))
        self._check(lib.phoebe_gpu_linewidths_rta_dev(self._ctx, C.byref(s), C.byref(nn), _ptr(k_index_dev),
                                                      _ptr(band_dev), _ptr(gamma_dev)))
        return nn.value

    def phonon_rates_elph(self, params, n_modes: int, **kw):
        """Phonon-electron rates P[q, nu] (eV) on the q grid of `params` (precision 7)."""
        s = params if isinstance(params, RTAParams) else make_params(params, **kw)
        nq = int(s.nq[0]) * int(s.nq[1]) * int(s.nq[2])
        out = np.empty((nq, int(n_modes)), dtype=np.float64)
        self._check(lib.phoebe_gpu_phonon_rates_elph(self._ctx, C.byref(s), C.c_int64(out.size), _ptr(out)))
        return out

    def transport_rta(self, params, lattice, **kw):
        """RTA sigma (S/m), Seebeck (V/K) and electronic kappa (W/(m K)), each 3 x 3."""
        s = params if isinstance(params, RTAParams) else make_params(params, **kw)
        lat = np.ascontiguousarray(lattice, dtype=np.float64).reshape(9)
        out = [np.empty(9) for _ in range(3)]
        self._check(lib.phoebe_gpu_transport_rta(self._ctx, C.byref(s), _ptr(lat), _ptr(out[0]), _ptr(out[1]),
                                                 _ptr(out[2])))
        return {"sigma": out[0].reshape(3, 3), "seebeck": out[1].reshape(3, 3), "kappa": out[2].reshape(3, 3)}

    def set_profiling(self, on: bool = True):
        self._check(lib.phoebe_gpu_set_profiling(self._ctx, 1 if on else 0))

    def set_memory_cap(self, nbytes: int):
        self._check(lib.phoebe_gpu_set_memory_cap(self._ctx, int(nbytes)))

    def stats(self) -> dict:
        s = Stats()
        self._check(lib.phoebe_gpu_get_stats(self._ctx, C.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    # -------------------------------------------------------------- learned q proposal
    def sampler_init(self, seed: int = 0):
        self._check(lib.phoebe_gpu_sampler_init(self._ctx, int(seed)))

    def sampler_load(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32).ravel()
        self._check(lib.phoebe_gpu_sampler_load(self._ctx, _ptr(a), a.size))

    def sampler_save(self) -> np.ndarray:
        a = np.empty(MLP_NPARAM, dtype=np.float32)
        self._check(lib.phoebe_gpu_sampler_save(self._ctx, _ptr(a), a.size))
        return a

    def sampler_train(self, grid_params, **opts) -> np.ndarray:
        """Train on one full-grid run; returns the mean loss of each epoch."""
        s = grid_params if isinstance(grid_params, RTAParams) else make_params(grid_params)
        o = TrainOpts()
        lib.phoebe_gpu_train_opts_default(C.byref(o))
        for key, val in opts.items():
            setattr(o, key, type(getattr(o, key))(val))
        loss = np.zeros(o.epochs)
        self._check(lib.phoebe_gpu_sampler_train(self._ctx, C.byref(s), C.byref(o), _ptr(loss)))
        return loss

    def q_contributions(self, params, nq_total: int | None = None, log_shell: bool = False, **kw):
        """c_nk(q) for every active state and q: returns (k_index, band, c [n][N_q] float32, features [n][4]),
        plus log phi [n][N_q] (the shell factor) with ``log_shell``."""
        s = params if isinstance(params, RTAParams) else make_params(params, **kw)
        n = C.c_int(0)
        self._check(lib.phoebe_gpu_q_contributions(self._ctx, C.byref(s), C.byref(n), None, None, None, None, None))
        Nq = int(s.nq[0]) * int(s.nq[1]) * int(s.nq[2])
        m = max(n.value, 1)
        ki = np.empty(m, dtype=np.int32)
        bd = np.empty(m, dtype=np.int32)
        cq = np.empty((m, Nq), dtype=np.float32)
        ft = np.empty((m, 4), dtype=np.float32)
        lp = np.empty((m, Nq), dtype=np.float32) if log_shell else None
        nn = C.c_int(m)
        self._check(lib.phoebe_gpu_q_contributions(self._ctx, C.byref(s), C.byref(nn), _ptr(ki), _ptr(bd), _ptr(cq),
                                                   _ptr(ft), _ptr(lp) if log_shell else None))
        k = nn.value
        if log_shell:
            return ki[:k], bd[:k], cq[:k], ft[:k], lp[:k]
        return ki[:k], bd[:k], cq[:k], ft[:k]

    def mlp_loss_grad(self, x, group_off=None, target=None, log_prior=None):
        """Network logits, and with targets the loss and gradient (softmax of z + log_prior), on explicit
        rows x [n][7]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        n = len(x)
        logits = np.empty(n, dtype=np.float32)
        if target is None:
            self._check(lib.phoebe_gpu_mlp_loss_grad(self._ctx, n, _ptr(x), 0, None, None, None, _ptr(logits), None,
                                                     None))
            return logits
        off = np.ascontiguousarray(group_off, dtype=np.int64)
        t = np.ascontiguousarray(target, dtype=np.float32)
        lp = None if log_prior is None else np.ascontiguousarray(log_prior, dtype=np.float32)
        loss = C.c_double(0.0)
        grad = np.empty(MLP_NPARAM, dtype=np.float32)
        self._check(lib.phoebe_gpu_mlp_loss_grad(self._ctx, n, _ptr(x), len(off) - 1, _ptr(off), _ptr(t),
                                                 None if lp is None else _ptr(lp), _ptr(logits), C.byref(loss),
                                                 _ptr(grad)))
        return logits, loss.value, grad

    def mlp_scores(self, features, nq, tensor_cores: bool = True) -> np.ndarray:
        """Network scores [n_states][N_q] of feature rows (eps - mu, v[3]) over every q of the grid nq."""
        f = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, 4)
        g = np.ascontiguousarray(nq, dtype=np.int32)
        z = np.empty((len(f), int(np.prod(g))), dtype=np.float32)
        self._check(lib.phoebe_gpu_mlp_scores(self._ctx, len(f), _ptr(f), _ptr(g), 1 if tensor_cores else 0, _ptr(z)))
        return z

    def is_uniforms(self, seed: int, k: int, n: int) -> np.ndarray:
        u = np.empty(int(n), dtype=np.float64)
        self._check(lib.phoebe_gpu_is_uniforms(self._ctx, int(seed), int(k), int(n), _ptr(u)))
        return u

    def fp32_rate(self) -> tuple:
        """Measured FP32 FMA rate of the device: (TFLOP/s, ms of the timed launch)."""
        t, ms = C.c_double(0.0), C.c_double(0.0)
        self._check(lib.phoebe_gpu_selftest_fp32_rate(self._ctx, C.byref(t), C.byref(ms)))
        return t.value, ms.value


def linewidths_rta_batch(jobs, capacities=None, **opts):
    """Linewidths of several materials in one call.

    ``jobs``: list of (PhoebeGPU context holding the material, params).  ``capacities``:
    optional upper bounds of each job's active-state count (skips the counting call).
    Returns (list of (k_index, band, gamma_eV) per job, dict of the batch timings and the
    stage-2 tile shape chosen per job)."""
    n = len(jobs)
    params = [p if isinstance(p, RTAParams) else make_params(p) for _, p in jobs]
    items = (BatchItem * n)()
    for i, (ctx, _) in enumerate(jobs):
        items[i].ctx = ctx._ctx.value
        items[i].params = C.cast(C.pointer(params[i]), C.c_void_p).value
    o = BatchOpts()
    lib.phoebe_gpu_batch_opts_default(C.byref(o))
    for key, val in opts.items():
        setattr(o, key, type(getattr(o, key))(val))

    def check(st):
        if st != 0:
            msgs = [lib.phoebe_gpu_last_error(ctx._ctx).decode() for ctx, _ in jobs]
            raise PhoebeGPUError(st, "; ".join(m for m in msgs if m) or "batch failed")
    if capacities is None:
        check(lib.phoebe_gpu_linewidths_rta_batch(items, n, C.byref(o)))     # counts
    outs = []
    for i in range(n):
        m = max(items[i].n_states if capacities is None else int(capacities[i]), 1)
        ki, bd, gm = np.empty(m, dtype=np.int32), np.empty(m, dtype=np.int32), np.empty(m)
        outs.append((ki, bd, gm))
        items[i].n_states = m
        items[i].k_index, items[i].band, items[i].gamma_eV = ki.ctypes.data, bd.ctypes.data, gm.ctypes.data
    check(lib.phoebe_gpu_linewidths_rta_batch(items, n, C.byref(o)))
    res = [(ki[:items[i].n_states], bd[:items[i].n_states], gm[:items[i].n_states]) for i, (ki, bd, gm) in
           enumerate(outs)]
    info = {name: getattr(o, name) for name, _ in BatchOpts._fields_ if name != "reserved"}
    info["tiles"] = [(items[i].tile_n, items[i].tile_kb) for i in range(n)]
    return res, info
