"""ctypes binding of libhubbard_ed.so (include/ed.h).

Argument marshalling only: every call goes straight to the C ABI, which runs
the whole path in the library's CUDA kernels.  Functions keep the C names.
Vectors may be torch tensors (CUDA or CPU), numpy arrays, or raw integer
addresses; CUDA tensors are passed as device pointers, host arrays as host
pointers (the library copies those itself).

If the library has not been built the import raises: there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ED_C128 = 0
ED_C64 = 1
ED_MIDPOINT = 0
ED_CFET4 = 1
ED_KERNEL_KINDS = 6
KERNEL_KIND_NAMES = ["apply", "update", "expm", "combine", "energy", "overlap"]

_STATUS = {0: "ED_OK", 1: "ED_ERR_ARG", 2: "ED_ERR_CUDA", 3: "ED_ERR_OOM",
           4: "ED_ERR_TIMEOUT", 5: "ED_ERR_UNSUPPORTED", 6: "ED_ERR_STATE",
           7: "ED_ERR_NUMERIC"}


class EDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


ED_PULSE_SIN_GAUSS = 0
ED_PULSE_COS_PHASE = 1


class ed_pulse(ctypes.Structure):
    _fields_ = [("A0", ctypes.c_double), ("omega", ctypes.c_double),
                ("sigma", ctypes.c_double), ("t0", ctypes.c_double),
                ("dir", ctypes.c_double * 3), ("b", ctypes.c_double),
                ("shape", ctypes.c_int), ("reserved", ctypes.c_int)]


class ed_observables(ctypes.Structure):
    _fields_ = [("docc", ctypes.c_void_p), ("norm2", ctypes.c_void_p),
                ("energy", ctypes.c_void_p), ("delta", ctypes.c_void_p),
                ("m_eff", ctypes.c_void_p), ("profile", ctypes.c_int32),
                ("kernel_ms", ctypes.c_void_p),
                ("kernel_launches", ctypes.c_void_p)]


def _load():
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_2005_13498_gb300.build` "
            "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    sig = {
        "ed_build_basis": [ctypes.POINTER(P), I, I, I],
        "ed_dims": [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
        "ed_get_basis": [P, I, P],
        "ed_set_lattice": [P, I, P, P, P, P, D, P],
        "ed_set_field": [P, P],
        "ed_get_table": [P, I, P, P, ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_int32)],
        "ed_apply_H": [P, P, P, I, I, P],
        "ed_ground_state": [P, P, ctypes.POINTER(D), D, I, ctypes.c_uint64,
                            ctypes.POINTER(D)],
        "ed_propagate": [P, P, I, ctypes.POINTER(ed_pulse), D, D, I, I,
                         ctypes.POINTER(ed_observables), P],
        "ed_double_occupation": [P, P, I, ctypes.POINTER(D), P],
        "ed_double_occupation_static": [P, P, I, ctypes.POINTER(D), P, P],
        "ed_spectral_propagate": [P, P, I, ctypes.POINTER(ed_pulse), D, I, I,
                                  P, P, P],
        "ed_apply_fermion_op": [P, P, I, I, I, P, P, I, P],
        "ed_spectral_propagate_at": [P, P, D, I, ctypes.POINTER(ed_pulse), D, I, I,
                                     P, P, P],
        "ed_spectral_function": [P, I, I, D, D, P, I, P],
        "ed_device_bytes": [P, ctypes.POINTER(ctypes.c_int64)],
        "ed_apply_config_info": [I] + [ctypes.POINTER(ctypes.c_int)] * 7,
        "ed_set_apply_config": [I],
        "ed_set_krylov_tol": [P, D],
        "ed_set_workspace_limit": [P, ctypes.c_int64],
        "ed_set_wait_fault": [I, ctypes.c_int64],
        "ed_set_integrator": [P, I],
        "ed_step_coefficients": [P, ctypes.POINTER(ed_pulse), D, D, I, P,
                                 ctypes.POINTER(ctypes.c_int), P],
        "ed_tridiag_expm": [I, I, P, P, D, P],
        "ed_get_apply_config": [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "ed_destroy": [P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ed_apply_config_count.argtypes = []
    lib.ed_apply_config_count.restype = ctypes.c_int
    lib.ed_last_error.argtypes = [P]
    lib.ed_last_error.restype = ctypes.c_char_p
    lib.ed_version.argtypes = []
    lib.ed_version.restype = ctypes.c_char_p
    return lib


lib = _load()


def _check(st, ctx=None):
    if st != 0:
        raise EDError(st, lib.ed_last_error(ctx).decode())


def ptr(x):
    """Address of a torch tensor / numpy array / int (no copies)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def ed_version():
    return lib.ed_version().decode()


def ed_build_basis(Ns, n_up, n_dn):
    h = ctypes.c_void_p()
    _check(lib.ed_build_basis(ctypes.byref(h), Ns, n_up, n_dn))
    return h.value


def ed_dims(ctx):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib.ed_dims(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def ed_get_basis(ctx, spin):
    du, dd = ed_dims(ctx)
    out = np.zeros(du if spin == 0 else dd, dtype=np.uint32)
    _check(lib.ed_get_basis(ctx, spin, ptr(out)), ctx)
    return out


def ed_set_lattice(ctx, lattice, U):
    """lattice: dict with Ns, p, q, t, d (n_bonds x 3), eps (or None)."""
    p = np.ascontiguousarray(lattice["p"], dtype=np.int32)
    q = np.ascontiguousarray(lattice["q"], dtype=np.int32)
    t = np.ascontiguousarray(lattice["t"], dtype=np.float64)
    d = np.ascontiguousarray(lattice["d"], dtype=np.float64).reshape(-1)
    eps = lattice.get("eps")
    eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    _check(lib.ed_set_lattice(ctx, len(p), ptr(p), ptr(q), ptr(t), ptr(d),
                              float(U), ptr(eps)), ctx)


def ed_set_field(ctx, A):
    a = np.ascontiguousarray(A, dtype=np.float64)
    _check(lib.ed_set_field(ctx, ptr(a)), ctx)


def ed_get_table(ctx, spin):
    nnz, ncl = ctypes.c_int64(), ctypes.c_int32()
    _check(lib.ed_get_table(ctx, spin, None, None, ctypes.byref(nnz),
                            ctypes.byref(ncl)), ctx)
    du, dd = ed_dims(ctx)
    off = np.zeros((du if spin == 0 else dd) + 1, dtype=np.int32)
    ent = np.zeros(max(1, nnz.value), dtype=np.uint32)
    _check(lib.ed_get_table(ctx, spin, ptr(off), ptr(ent), ctypes.byref(nnz),
                            ctypes.byref(ncl)), ctx)
    return off, ent[:nnz.value], ncl.value


def ed_apply_H(ctx, v, w, dtype, nvec=1, stream=None):
    _check(lib.ed_apply_H(ctx, ptr(v), ptr(w), dtype, nvec, stream_ptr(stream)), ctx)


def ed_ground_state(ctx, psi, tol=1e-12, max_iter=2000, seed=1):
    E0, res = ctypes.c_double(), ctypes.c_double()
    _check(lib.ed_ground_state(ctx, ptr(psi), ctypes.byref(E0), tol, max_iter,
                               seed, ctypes.byref(res)), ctx)
    return E0.value, res.value


def make_pulse(p):
    """dict(A0, omega, sigma, t0, dir[, shape "sin" | "cos_phase", b])."""
    if p is None:
        return None
    shape = {"sin": ED_PULSE_SIN_GAUSS, "cos_phase": ED_PULSE_COS_PHASE}[p.get("shape", "sin")]
    return ed_pulse(p["A0"], p["omega"], p["sigma"], p["t0"],
                    (ctypes.c_double * 3)(*p["dir"]), float(p.get("b", 0.0)), shape, 0)


def ed_propagate(ctx, psi, dtype, pulse, t_start, dt, n_steps, m,
                 energy=False, profile=False, stream=None):
    """Returns dict of numpy arrays: docc, norm2, energy, delta, m_eff, and
    kernel_ms / kernel_launches when profile is set."""
    out = {
        "docc": np.zeros(n_steps + 1), "norm2": np.zeros(n_steps + 1),
        "energy": np.zeros(n_steps + 1) if energy else None,
        "delta": np.zeros(max(1, n_steps)), "m_eff": np.zeros(max(1, n_steps), np.int32),
        "kernel_ms": np.zeros(ED_KERNEL_KINDS),
        "kernel_launches": np.zeros(ED_KERNEL_KINDS, np.int64),
    }
    obs = ed_observables(ptr(out["docc"]), ptr(out["norm2"]), ptr(out["energy"]),
                         ptr(out["delta"]), ptr(out["m_eff"]), 1 if profile else 0,
                         ptr(out["kernel_ms"]), ptr(out["kernel_launches"]))
    pl = make_pulse(pulse)
    _check(lib.ed_propagate(ctx, ptr(psi), dtype,
                            ctypes.byref(pl) if pl is not None else None,
                            float(t_start), float(dt), int(n_steps), int(m),
                            ctypes.byref(obs), stream_ptr(stream)), ctx)
    out["delta"] = out["delta"][:n_steps]
    out["m_eff"] = out["m_eff"][:n_steps]
    return out


def ed_double_occupation(ctx, psi, dtype, Ns=None):
    d = ctypes.c_double()
    du, dd = ed_dims(ctx)
    site = np.zeros(16)
    _check(lib.ed_double_occupation(ctx, ptr(psi), dtype, ctypes.byref(d),
                                    ptr(site)), ctx)
    return d.value, site


def ed_double_occupation_static(ctx, psi, dtype, stream=None):
    """Same results as ed_double_occupation, with no device allocation
    (scratch in a fixed library array; psi must be on the device)."""
    d = ctypes.c_double()
    site = np.zeros(16)
    _check(lib.ed_double_occupation_static(ctx, ptr(psi), dtype, ctypes.byref(d),
                                           ptr(site), stream_ptr(stream)), ctx)
    return d.value, site


def ed_spectral_propagate(ctx, psi0, dtype, pulse, dt, n_steps, m, Ns,
                          stream=None):
    """Returns (G_less, G_greater) complex arrays [n_steps+1, Ns, 2]."""
    gl = np.zeros((n_steps + 1, Ns, 2, 2))
    gg = np.zeros((n_steps + 1, Ns, 2, 2))
    pl = make_pulse(pulse)
    _check(lib.ed_spectral_propagate(ctx, ptr(psi0), dtype,
                                     ctypes.byref(pl) if pl is not None else None,
                                     float(dt), int(n_steps), int(m), ptr(gl),
                                     ptr(gg), stream_ptr(stream)), ctx)
    return gl[..., 0] + 1j * gl[..., 1], gg[..., 0] + 1j * gg[..., 1]


def ed_spectral_propagate_at(ctx, psi_ref, t_ref, dtype, pulse, dt, n_steps, m, Ns,
                             stream=None):
    """Green's functions at (t_ref, t_ref + n dt); psi_ref = psi(t_ref)."""
    gl = np.zeros((n_steps + 1, Ns, 2, 2))
    gg = np.zeros((n_steps + 1, Ns, 2, 2))
    pl = make_pulse(pulse)
    _check(lib.ed_spectral_propagate_at(ctx, ptr(psi_ref), float(t_ref), dtype,
                                        ctypes.byref(pl) if pl is not None else None,
                                        float(dt), int(n_steps), int(m), ptr(gl),
                                        ptr(gg), stream_ptr(stream)), ctx)
    return gl[..., 0] + 1j * gl[..., 1], gg[..., 0] + 1j * gg[..., 1]


def ed_spectral_function(G, dt, eps, nu):
    """(1/pi) Im int_0^T e^{-eps t} e^{i nu t} G(t) dt (trapezoid) for G of
    shape [n_steps+1, ...] (complex); returns [len(nu), ...]."""
    G = np.asarray(G, dtype=np.complex128)
    shp = G.shape[1:]
    nser = int(np.prod(shp)) if shp else 1
    g = np.ascontiguousarray(np.stack([G.real, G.imag], axis=-1).reshape(G.shape[0], nser, 2))
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    A = np.zeros((len(nu), nser))
    _check(lib.ed_spectral_function(ptr(g), G.shape[0] - 1, nser, float(dt), float(eps),
                                    ptr(nu), len(nu), ptr(A)))
    return A.reshape((len(nu),) + shp)


def ed_apply_fermion_op(ctx, ctx_dst, site, spin, create, psi, out, dtype,
                        stream=None):
    _check(lib.ed_apply_fermion_op(ctx, ctx_dst, site, spin, 1 if create else 0,
                                   ptr(psi), ptr(out), dtype, stream_ptr(stream)), ctx)


def ed_set_krylov_tol(ctx, tol):
    """0: fixed Krylov dimension m (default); > 0: adaptive exit of
    Algorithm 6 with m as the maximum."""
    _check(lib.ed_set_krylov_tol(ctx, float(tol)), ctx)


def ed_set_workspace_limit(ctx, nbytes):
    """Cap (bytes) on the Krylov workspace of the context's propagations and
    ground-state solves; 0 = no cap."""
    _check(lib.ed_set_workspace_limit(ctx, int(nbytes)), ctx)


def ed_set_wait_fault(withhold_copy=-1, wait_polls=0):
    """Test hook of the bounded device-side waits (process-wide): the T_up
    copy the TMA producer stops at (-1: none) and the poll limit (0: default)."""
    _check(lib.ed_set_wait_fault(int(withhold_copy), int(wait_polls)))


def ed_set_integrator(ctx, scheme):
    """ED_MIDPOINT (Eq. (32), default) or ED_CFET4 (fourth order, two Krylov
    steps of dt/2 per time step); also accepts "midpoint" / "cfet4"."""
    if isinstance(scheme, str):
        scheme = {"midpoint": ED_MIDPOINT, "cfet4": ED_CFET4}[scheme]
    _check(lib.ed_set_integrator(ctx, int(scheme)), ctx)


def ed_step_coefficients(ctx, n_bonds, pulse, t_start, dt, n_steps):
    """(coef[n_sub, n_bonds] complex: the hop p_b -> q_b of every Krylov
    sub-step, tau of a sub-step)."""
    pp = make_pulse(pulse)
    pref = ctypes.byref(pp) if pp is not None else None
    n_sub, tau = ctypes.c_int(), ctypes.c_double()
    _check(lib.ed_step_coefficients(ctx, pref, float(t_start), float(dt), int(n_steps), None,
                                    ctypes.byref(n_sub), ctypes.byref(tau)), ctx)
    out = np.zeros((n_sub.value, n_bonds), dtype=np.complex128)
    _check(lib.ed_step_coefficients(ctx, pref, float(t_start), float(dt), int(n_steps),
                                    out.ctypes.data, None, None), ctx)
    return out, tau.value


def ed_tridiag_expm(alpha, beta, tau):
    """y = exp(-i tau T) e_1 for a batch of tridiagonals: alpha [batch, n],
    beta [batch, n-1] (float64) -> y [batch, n] complex128, on the GPU."""
    a = np.ascontiguousarray(np.atleast_2d(alpha), dtype=np.float64)
    batch, n = a.shape
    b = np.ascontiguousarray(np.reshape(beta, (batch, max(0, n - 1))), dtype=np.float64)
    y = np.zeros((batch, n), dtype=np.complex128)
    _check(lib.ed_tridiag_expm(batch, n, a.ctypes.data, b.ctypes.data if n > 1 else None,
                               float(tau), y.ctypes.data))
    return y


def ed_apply_config_count():
    return lib.ed_apply_config_count()


def ed_apply_config_info(config):
    """dict(fp64, rows_per_cta, pairs_per_thread, ctas_per_sm, split, tma, mv)."""
    v = [ctypes.c_int() for _ in range(7)]
    _check(lib.ed_apply_config_info(config, *[ctypes.byref(x) for x in v]))
    keys = ["fp64", "rows_per_cta", "pairs_per_thread", "ctas_per_sm", "split", "tma", "mv"]
    return {k: x.value for k, x in zip(keys, v)}


def ed_set_apply_config(config):
    """-1: autotune (default); otherwise pin the H v configuration."""
    _check(lib.ed_set_apply_config(int(config)))


def ed_get_apply_config(ctx):
    """(propagation engine configuration, ed_apply_H plan configuration)."""
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(lib.ed_get_apply_config(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


def ed_device_bytes(ctx):
    b = ctypes.c_int64()
    _check(lib.ed_device_bytes(ctx, ctypes.byref(b)), ctx)
    return b.value


def ed_destroy(ctx):
    lib.ed_destroy(ctx)


def ed_last_error(ctx=None):
    return lib.ed_last_error(ctx).decode()


class Hubbard:
    """Owning wrapper: one context (sector) with its lattice."""

    def __init__(self, lattice, n_up, n_dn, U):
        self.Ns = lattice["Ns"]
        self.n_up, self.n_dn, self.U = n_up, n_dn, U
        self.ctx = ed_build_basis(self.Ns, n_up, n_dn)
        ed_set_lattice(self.ctx, lattice, U)
        self.dim_up, self.dim_dn = ed_dims(self.ctx)
        self.D = self.dim_up * self.dim_dn

    def close(self):
        if self.ctx:
            ed_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
