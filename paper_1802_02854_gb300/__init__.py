"""GB300 FTKomega hot path: Python binding of the C-ABI in include/ftk.h.

The binding only marshals arguments: every step of the path runs in the
CUDA kernels of libftk.so (paper_1802_02854_gb300/csrc). There is no CPU
fallback: if the library is missing, importing works but every call raises
FtkError telling how to build it. PyTorch provides device memory (the
workspace tensor) and streams.

Low-level functions carry the C names (ftk_create, ftk_tpq_step, ...);
``Context`` bundles a context with its workspace tensor.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libftk.so")

FTK_OK, FTK_EINVAL, FTK_ENOMEM, FTK_ECUDA, FTK_ENOCONV, FTK_EBREAKDOWN, FTK_ETIMEOUT, FTK_ETRUNC, FTK_EBUSY = range(9)
FTK_FP64, FTK_FP32, FTK_MIXED, FTK_DF = 0, 1, 2, 3
PRECISIONS = {"fp64": FTK_FP64, "fp32": FTK_FP32, "mixed": FTK_MIXED, "df": FTK_DF}
STATUS_NAMES = ["FTK_OK", "FTK_EINVAL", "FTK_ENOMEM", "FTK_ECUDA", "FTK_ENOCONV", "FTK_EBREAKDOWN",
                "FTK_ETIMEOUT", "FTK_ETRUNC", "FTK_EBUSY"]

# Every symbol declared in include/ftk.h.
EXPORTS = ["ftk_footprint", "ftk_create", "ftk_bind_workspace", "ftk_tpq_init", "ftk_set_state",
           "ftk_tpq_step", "ftk_shells", "ftk_apply_op", "ftk_set_probe", "ftk_shifted_cocg",
           "ftk_spectrum", "ftk_hv", "ftk_get_vector", "ftk_plan_info", "ftk_launch_count",
           "ftk_last_error", "ftk_destroy", "ftk_tpq_step_noalloc", "ftk_suggest_order", "ftk_autotune", "ftk_set_relax",
           "ftk_shifted_cocg_ex", "ftk_ctpq", "ftk_filter_footprint", "ftk_filter_shells", "ftk_filter_spectrum",
           "ftk_spectrum_ex", "ftk_sector_create", "ftk_sector_destroy", "ftk_sector_info", "ftk_sector_set",
           "ftk_sector_get", "ftk_sector_project", "ftk_sector_hv", "ftk_sector_tpq", "ftk_sector_apply_sz",
           "ftk_sector_green", "ftk_sector_combine"]


class FtkError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class _Lattice(C.Structure):
    _fields_ = [("n_sites", C.c_int32), ("pos", C.POINTER(C.c_double))]


class _Bond(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("gamma", C.c_int32)]


class _Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_rhs", C.c_int32), ("n_saved", C.c_int32),
                ("tile_bits", C.c_int32), ("cuda_stream", C.c_void_p)]


class _CocgOpts(C.Structure):
    _fields_ = [("proj_slots", C.POINTER(C.c_int32)), ("seed_index", C.c_int32), ("seed_switch", C.c_int32)]


_lib = None


def lib() -> C.CDLL:
    """Load libftk.so (built by paper_1802_02854_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FtkError(FTK_ECUDA, f"{LIB_PATH} not built; run paper_1802_02854_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    pd = C.POINTER(C.c_double)
    pi = C.POINTER(C.c_int32)
    L.ftk_footprint.argtypes = [i32, i32, i32, i32]
    L.ftk_footprint.restype = C.c_size_t
    L.ftk_create.argtypes = [C.POINTER(_Lattice), C.POINTER(_Bond), i32, dbl, dbl, C.POINTER(_Opts), C.POINTER(vp)]
    L.ftk_bind_workspace.argtypes = [vp, vp, C.c_size_t]
    L.ftk_tpq_init.argtypes = [vp, C.c_uint64, C.c_uint32, dbl]
    L.ftk_set_state.argtypes = [vp, vp, i32, dbl]
    L.ftk_tpq_step.argtypes = [vp, i32, i32, pd, pd, pd]
    L.ftk_shells.argtypes = [vp, pi, pi, pd]
    L.ftk_apply_op.argtypes = [vp, i32, i32, pd, i32]
    L.ftk_set_probe.argtypes = [vp, i32, vp, i32, dbl]
    L.ftk_shifted_cocg.argtypes = [vp, pi, i32, pd, i32, dbl, dbl, i32, pd, pi]
    L.ftk_spectrum.argtypes = [vp, pd, i32, i32, pd, i32, pd, pi]
    L.ftk_hv.argtypes = [vp, vp, vp, i32]
    L.ftk_get_vector.argtypes = [vp, i32, pd]
    L.ftk_plan_info.argtypes = [vp, pi, pi]
    L.ftk_launch_count.argtypes = [vp]
    L.ftk_launch_count.restype = i64
    L.ftk_last_error.argtypes = [vp]
    L.ftk_last_error.restype = C.c_char_p
    L.ftk_destroy.argtypes = [vp]
    L.ftk_destroy.restype = None
    L.ftk_tpq_step_noalloc.argtypes = [i32, C.POINTER(_Bond), i32, dbl, dbl, dbl, vp, vp, pd, vp]
    L.ftk_suggest_order.argtypes = [i32, C.POINTER(_Bond), i32, i32, i32, i32, pi, pi]
    L.ftk_autotune.argtypes = [vp, i32, i32, pi, pi, pd]
    L.ftk_set_relax.argtypes = [vp, C.c_double]
    L.ftk_shifted_cocg_ex.argtypes = [vp, pi, i32, pd, i32, dbl, i32, C.POINTER(_CocgOpts), pd, pi, pi]
    L.ftk_ctpq.argtypes = [vp, pd, i32, dbl, i32, pd, pi, pd]
    L.ftk_filter_footprint.argtypes = [i32, i32, i32]
    L.ftk_filter_footprint.restype = C.c_size_t
    L.ftk_filter_shells.argtypes = [vp, i32, dbl, dbl, i32, i32, dbl, i32, vp, C.c_size_t, i32, pd, pi]
    L.ftk_filter_spectrum.argtypes = [vp, pd, i32, i32, pd, pd, dbl, dbl, pd, i32, pd, pd]
    L.ftk_spectrum_ex.argtypes = [vp, pd, i32, i32, pd, i32, pd, pd, i32, i32, dbl, pd, pi]
    L.ftk_sector_create.argtypes = [vp, pi, i32, pd, i32, C.POINTER(vp), C.POINTER(i64)]
    L.ftk_sector_destroy.argtypes = [vp]
    L.ftk_sector_destroy.restype = None
    L.ftk_sector_info.argtypes = [vp, C.POINTER(i64), pi, C.POINTER(C.c_uint32)]
    L.ftk_sector_set.argtypes = [vp, i32, vp, i32]
    L.ftk_sector_get.argtypes = [vp, i32, pd]
    L.ftk_sector_project.argtypes = [vp, vp, i32, i32]
    L.ftk_sector_hv.argtypes = [vp, i32, i32]
    L.ftk_sector_tpq.argtypes = [vp, i32, i32, dbl, i32, i32, i32, pd, pd, pd]
    L.ftk_sector_apply_sz.argtypes = [vp, i32, vp, i32, pd]
    L.ftk_sector_green.argtypes = [vp, i32, pd, i32, dbl, i32, pd, pi]
    L.ftk_sector_combine.argtypes = [i32, i32, pd, pd, pd, i32, pi, i32, pd, pd, pd, pd]
    for name in EXPORTS:
        if name not in ("ftk_footprint", "ftk_launch_count", "ftk_last_error", "ftk_destroy", "ftk_filter_footprint",
                        "ftk_sector_destroy"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32)) if a is not None else None


def _check(ctx, st, ok=(FTK_OK,)):
    if st not in ok:
        msg = lib().ftk_last_error(ctx).decode()
        raise FtkError(st, msg)
    return st


# ----------------------------------------------------------- C-named wrappers
def ftk_footprint(n_sites, n_saved, max_rhs, precision):
    return int(lib().ftk_footprint(n_sites, n_saved, max_rhs, precision))


def ftk_create(n_sites, pos, bonds, K, J, precision=FTK_FP64, max_rhs=1, n_saved=1, tile_bits=0,
               stream=None):
    """pos: float64 [N, 2]; bonds: int [n_bonds, 3] rows (i, j, gamma). Returns the context handle."""
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1)
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 3)
    lat = _Lattice(int(n_sites), pos.ctypes.data_as(C.POINTER(C.c_double)))
    barr = (_Bond * len(bonds))(*[_Bond(int(i), int(j), int(g)) for i, j, g in bonds])
    opts = _Opts(int(precision), int(max_rhs), int(n_saved), int(tile_bits),
                 C.c_void_p(int(stream) if stream else 0))
    out = C.c_void_p()
    st = lib().ftk_create(C.byref(lat), barr, len(bonds), float(K), float(J), C.byref(opts), C.byref(out))
    _check(None, st)
    return out.value


def ftk_bind_workspace(ctx, dev_ptr, nbytes):
    _check(ctx, lib().ftk_bind_workspace(ctx, C.c_void_p(dev_ptr), nbytes))


def ftk_tpq_init(ctx, seed, sample, ell):
    _check(ctx, lib().ftk_tpq_init(ctx, seed, sample, ell))


def ftk_set_state(ctx, v, ell):
    """v: complex128 host array (numpy) or a device pointer (int)."""
    if isinstance(v, int):
        _check(ctx, lib().ftk_set_state(ctx, C.c_void_p(v), 1, ell))
    else:
        a = np.ascontiguousarray(v, dtype=np.complex128)
        _check(ctx, lib().ftk_set_state(ctx, a.ctypes.data_as(C.c_void_p), 0, ell))


def ftk_tpq_step(ctx, n_steps, save_every):
    u = np.zeros(n_steps)
    lq = np.zeros(n_steps)
    h2 = np.zeros(n_steps)
    _check(ctx, lib().ftk_tpq_step(ctx, n_steps, save_every, _dp(u), _dp(lq), _dp(h2)))
    return u, lq, h2


def ftk_shells(ctx, cap=4096):
    n = C.c_int32()
    steps = np.zeros(cap, dtype=np.int32)
    en = np.zeros(cap)
    _check(ctx, lib().ftk_shells(ctx, C.byref(n), _ip(steps), _dp(en)))
    return steps[: n.value].copy(), en[: n.value].copy()


def ftk_apply_op(ctx, shell, gamma, q, slot):
    qq = np.ascontiguousarray(q, dtype=np.float64)
    _check(ctx, lib().ftk_apply_op(ctx, shell, gamma, _dp(qq), slot))


def ftk_set_probe(ctx, slot, v, energy):
    if isinstance(v, int):
        _check(ctx, lib().ftk_set_probe(ctx, slot, C.c_void_p(v), 1, energy))
    else:
        a = np.ascontiguousarray(v, dtype=np.complex128)
        _check(ctx, lib().ftk_set_probe(ctx, slot, a.ctypes.data_as(C.c_void_p), 0, energy))


def ftk_shifted_cocg(ctx, slots, omega, eta, tol, max_iter, allow_noconv=False):
    """Returns (G complex128 [n_rhs, n_omega], iters int32 [n_rhs], status)."""
    sl = np.ascontiguousarray(slots, dtype=np.int32)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    G = np.zeros((len(sl), len(om)), dtype=np.complex128)
    it = np.zeros(len(sl), dtype=np.int32)
    ok = (FTK_OK, FTK_ENOCONV) if allow_noconv else (FTK_OK,)
    st = _check(ctx, lib().ftk_shifted_cocg(ctx, _ip(sl), len(sl), _dp(om), len(om), eta, tol, max_iter,
                                            G.ctypes.data_as(C.POINTER(C.c_double)), _ip(it)), ok)
    return G, it, st


def ftk_shifted_cocg_ex(ctx, slots, shifts, tol, max_iter, proj_slots=None, seed_index=-1, seed_switch=False,
                        allow_noconv=False):
    """General complex shifts z_s = E_j + shifts[s] (Im > 0), optional
    projection slots (A != B) and seed switching. Returns (G [n_rhs, n_shift],
    iters [n_rhs], switches [n_rhs], status)."""
    sl = np.ascontiguousarray(slots, dtype=np.int32)
    z = np.ascontiguousarray(shifts, dtype=np.complex128)
    G = np.zeros((len(sl), len(z)), dtype=np.complex128)
    it = np.zeros(len(sl), dtype=np.int32)
    sw = np.zeros(len(sl), dtype=np.int32)
    pj = None if proj_slots is None else np.ascontiguousarray(proj_slots, dtype=np.int32)
    opts = _CocgOpts(_ip(pj) if pj is not None else None, int(seed_index), 1 if seed_switch else 0)
    ok = (FTK_OK, FTK_ENOCONV) if allow_noconv else (FTK_OK,)
    st = _check(ctx, lib().ftk_shifted_cocg_ex(ctx, _ip(sl), len(sl), z.ctypes.data_as(C.POINTER(C.c_double)),
                                               len(z), float(tol), int(max_iter), C.byref(opts),
                                               G.ctypes.data_as(C.POINTER(C.c_double)), _ip(it), _ip(sw)), ok)
    return G, it, sw, st


def ftk_ctpq(ctx, betas, lam=1e4, first_shell=0):
    """cTPQ states at the ascending betas (Appendix A), kept as shells
    first_shell.. Returns (log norms, M_d per increment, energies)."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    ln = np.zeros(len(b))
    md = np.zeros(len(b), dtype=np.int32)
    en = np.zeros(len(b))
    _check(ctx, lib().ftk_ctpq(ctx, _dp(b), len(b), float(lam), int(first_shell), _dp(ln), _ip(md), _dp(en)))
    return ln, md, en


def ftk_filter_footprint(n_centres, n_points, max_iter):
    return int(lib().ftk_filter_footprint(int(n_centres), int(n_points), int(max_iter)))


def ftk_filter_shells(ctx, src, e_b, eps, n_centres, n_points, tol, max_iter, scratch_ptr, scratch_bytes,
                      first_shell=0):
    """Filtered shells P_{E_m, eps, M} phi (Sec. II.C) into shells
    first_shell..; returns (norms <phi^m|phi^m> [L], iterations)."""
    n2 = np.zeros(int(n_centres))
    it = C.c_int32()
    _check(ctx, lib().ftk_filter_shells(ctx, int(src), float(e_b), float(eps), int(n_centres), int(n_points),
                                        float(tol), int(max_iter), C.c_void_p(scratch_ptr), int(scratch_bytes),
                                        int(first_shell), _dp(n2), C.byref(it)))
    return n2, it.value


def ftk_filter_spectrum(ctx, G, energy, norm2, beta, eps, T):
    """Eqs. FRW1/FRW2: returns (S [n_T, n_omega], P [n_T, n_shell])."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    E = np.ascontiguousarray(energy, dtype=np.float64)
    N2 = np.ascontiguousarray(norm2, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    S = np.zeros((len(T), G.shape[1]))
    P = np.zeros((len(T), G.shape[0]))
    _check(ctx, lib().ftk_filter_spectrum(ctx, G.ctypes.data_as(C.POINTER(C.c_double)), G.shape[0], G.shape[1],
                                          _dp(E), _dp(N2), float(beta), float(eps), _dp(T), len(T), _dp(S),
                                          _dp(P)))
    return S, P


def ftk_spectrum_ex(ctx, G, T, u, logQ, save_every, ell):
    """R1 reweighting with caller statistics; returns (S [n_T, n_omega], trunc [n_T])."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    T = np.ascontiguousarray(T, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    lq = np.ascontiguousarray(logQ, dtype=np.float64)
    S = np.zeros((len(T), G.shape[1]))
    tr = np.zeros(len(T), dtype=np.int32)
    _check(ctx, lib().ftk_spectrum_ex(ctx, G.ctypes.data_as(C.POINTER(C.c_double)), G.shape[0], G.shape[1], _dp(T),
                                      len(T), _dp(u), _dp(lq), len(u), int(save_every), float(ell), _dp(S), _ip(tr)),
           (FTK_OK, FTK_ETRUNC))
    return S, tr


def ftk_sector_combine(lognorm0, logq, u, shell_steps=None, G=None):
    """Merge sector statistics (and per-sector shell Green's functions
    G [n_sec, n_shell, n_omega]); returns (u, logQ, G or None)."""
    ln = np.ascontiguousarray(lognorm0, dtype=np.float64)
    lq = np.ascontiguousarray(logq, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    n_sec, n_steps = lq.shape
    uo = np.zeros(n_steps)
    lo = np.zeros(n_steps)
    if G is None:
        _check(None, lib().ftk_sector_combine(n_sec, n_steps, _dp(ln), _dp(lq), _dp(uu), 0, None, 0, None, _dp(uo),
                                              _dp(lo), None))
        return uo, lo, None
    Gs = np.ascontiguousarray(G, dtype=np.complex128)
    st = np.ascontiguousarray(shell_steps, dtype=np.int32)
    Go = np.zeros(Gs.shape[1:], dtype=np.complex128)
    _check(None, lib().ftk_sector_combine(n_sec, n_steps, _dp(ln), _dp(lq), _dp(uu), Gs.shape[1], _ip(st),
                                          Gs.shape[2], Gs.ctypes.data_as(C.POINTER(C.c_double)), _dp(uo), _dp(lo),
                                          Go.ctypes.data_as(C.POINTER(C.c_double))))
    return uo, lo, Go


class Sector:
    """A momentum sector of a context (translation group perms [n_g, N] and
    character chi [n_g] complex); owns its device memory."""

    def __init__(self, ctx, perms, chi, n_slots=8):
        self.ctx = ctx
        P = np.ascontiguousarray(perms, dtype=np.int32)
        ch = np.ascontiguousarray(chi, dtype=np.complex128)
        h = C.c_void_p()
        d = C.c_int64()
        _check(ctx.handle, lib().ftk_sector_create(ctx.handle, _ip(P), P.shape[0],
                                                   ch.ctypes.data_as(C.POINTER(C.c_double)), int(n_slots),
                                                   C.byref(h), C.byref(d)))
        self.handle = h.value
        self.dim = int(d.value)
        self.n_slots = n_slots

    def info(self):
        d = C.c_int64()
        no = C.c_int32()
        reps = np.zeros(self.dim, dtype=np.uint32)
        _check(self.ctx.handle, lib().ftk_sector_info(self.handle, C.byref(d), C.byref(no),
                                                      reps.ctypes.data_as(C.POINTER(C.c_uint32))))
        return int(d.value), int(no.value), reps

    def set(self, slot, v):
        a = np.ascontiguousarray(v, dtype=np.complex128)
        _check(self.ctx.handle, lib().ftk_sector_set(self.handle, int(slot), a.ctypes.data_as(C.c_void_p), 0))

    def get(self, slot):
        out = np.zeros(self.dim, dtype=np.complex128)
        _check(self.ctx.handle, lib().ftk_sector_get(self.handle, int(slot), out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def project(self, psi, slot):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        _check(self.ctx.handle, lib().ftk_sector_project(self.handle, a.ctypes.data_as(C.c_void_p), 0, int(slot)))

    def hv(self, slot_in, slot_out):
        _check(self.ctx.handle, lib().ftk_sector_hv(self.handle, int(slot_in), int(slot_out)))
        self.ctx.stream.synchronize()

    def tpq(self, slot_state, slot_work, ell, n_steps, save_every, first_save_slot):
        u = np.zeros(n_steps)
        lq = np.zeros(n_steps)
        l0 = C.c_double()
        _check(self.ctx.handle, lib().ftk_sector_tpq(self.handle, int(slot_state), int(slot_work), float(ell),
                                                     int(n_steps), int(save_every), int(first_save_slot), _dp(u),
                                                     _dp(lq), C.byref(l0)))
        return u, lq, l0.value

    def apply_sz(self, slot_src, dst, slot_dst, q):
        qq = np.ascontiguousarray(q, dtype=np.float64)
        _check(self.ctx.handle, lib().ftk_sector_apply_sz(self.handle, int(slot_src), dst.handle, int(slot_dst),
                                                          _dp(qq)))

    def green(self, slot, shifts, tol=1e-10, max_iter=10000, allow_noconv=False):
        z = np.ascontiguousarray(shifts, dtype=np.complex128)
        G = np.zeros(len(z), dtype=np.complex128)
        it = C.c_int32()
        ok = (FTK_OK, FTK_ENOCONV) if allow_noconv else (FTK_OK,)
        _check(self.ctx.handle, lib().ftk_sector_green(self.handle, int(slot), z.ctypes.data_as(C.POINTER(C.c_double)),
                                                       len(z), float(tol), int(max_iter),
                                                       G.ctypes.data_as(C.POINTER(C.c_double)), C.byref(it)), ok)
        return G, it.value

    def close(self):
        if self.handle:
            lib().ftk_sector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ftk_spectrum(ctx, G, T):
    """G: complex128 [n_shell, n_omega]; returns (S [n_T, n_omega], trunc [n_T])."""
    G = np.ascontiguousarray(G, dtype=np.complex128)
    T = np.ascontiguousarray(T, dtype=np.float64)
    S = np.zeros((len(T), G.shape[1]))
    tr = np.zeros(len(T), dtype=np.int32)
    _check(ctx, lib().ftk_spectrum(ctx, G.ctypes.data_as(C.POINTER(C.c_double)), G.shape[0], G.shape[1],
                                   _dp(T), len(T), _dp(S), _ip(tr)), (FTK_OK, FTK_ETRUNC))
    return S, tr


def ftk_hv(ctx, v_ptr, out_ptr, n_rhs):
    _check(ctx, lib().ftk_hv(ctx, C.c_void_p(v_ptr), C.c_void_p(out_ptr), n_rhs))


def ftk_get_vector(ctx, which, dim):
    out = np.zeros(dim, dtype=np.complex128)
    _check(ctx, lib().ftk_get_vector(ctx, which, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def ftk_plan_info(ctx):
    n = C.c_int32()
    b = C.c_int32()
    _check(ctx, lib().ftk_plan_info(ctx, C.byref(n), C.byref(b)))
    return n.value, b.value


def ftk_launch_count(ctx):
    return int(lib().ftk_launch_count(ctx))


def ftk_destroy(ctx):
    if ctx:
        lib().ftk_destroy(ctx)


def ftk_tpq_step_noalloc(n_sites, bonds, K, J, ell, psi_ptr, out_ptr, stream=None):
    """One allocation-free mTPQ step on caller device vectors (FP64).
    Returns (u, <H^2>, q); out = (l - H/N) psi unnormalised."""
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 3)
    barr = (_Bond * len(bonds))(*[_Bond(int(i), int(j), int(g)) for i, j, g in bonds])
    st = np.zeros(3)
    _check(None, lib().ftk_tpq_step_noalloc(int(n_sites), barr, len(bonds), float(K), float(J), float(ell),
                                            C.c_void_p(psi_ptr), C.c_void_p(out_ptr), _dp(st),
                                            C.c_void_p(int(stream) if stream else 0)))
    return float(st[0]), float(st[1]), float(st[2])


def ftk_autotune(ctx, n_rhs, which=0):
    """Time the admissible H.v plans for n_rhs vectors and install the
    fastest. Returns (tile_bits, cols, us per H.v)."""
    tb = C.c_int32()
    cols = C.c_int32()
    us = C.c_double()
    _check(ctx, lib().ftk_autotune(ctx, int(n_rhs), int(which), C.byref(tb), C.byref(cols), C.byref(us)))
    return tb.value, cols.value, us.value


def ftk_set_relax(ctx, theta):
    """Relaxed double-float solve threshold theta (0: off); FTK_DF contexts."""
    _check(ctx, lib().ftk_set_relax(ctx, float(theta)))


def ftk_suggest_order(n_sites, bonds, precision=FTK_FP64, n_rhs=1, tile_bits=0):
    """Site relabelling for fewer H.v passes: returns (perm, n_passes) with
    site l -> new label perm[l] (apply with ftk_inputs.relabel)."""
    bonds = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 3)
    barr = (_Bond * len(bonds))(*[_Bond(int(i), int(j), int(g)) for i, j, g in bonds])
    perm = np.zeros(n_sites, dtype=np.int32)
    npass = C.c_int32()
    _check(None, lib().ftk_suggest_order(int(n_sites), barr, len(bonds), int(precision), int(n_rhs),
                                         int(tile_bits), _ip(perm), C.byref(npass)))
    return perm.astype(np.int64), npass.value


# ----------------------------------------------------------------- wrapper
class Context:
    """A context plus the torch device workspace it runs in.

    cluster: object with n_sites, pos [N, 2], bonds [n_bonds, 3].
    precision: "fp64", "fp32", "mixed" (FP32 H.v, FP64 Krylov vectors) or "df"
    (double-float H.v on the FP32 pipe, FP64 Krylov vectors).
    stream: torch.cuda.Stream (default: a new one).
    """

    def __init__(self, cluster, K, J, precision="fp64", max_rhs=1, n_saved=1, tile_bits=0, stream=None,
                 workspace=None):
        import torch

        self.torch = torch
        self.n = int(cluster.n_sites)
        self.dim = 1 << self.n
        self.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.max_rhs = max_rhs
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.handle = ftk_create(self.n, cluster.pos, cluster.bonds, K, J, self.prec, max_rhs, n_saved,
                                 tile_bits, self.stream.cuda_stream)
        self.bytes = ftk_footprint(self.n, n_saved, max_rhs, self.prec)
        if workspace is None:
            workspace = torch.empty(self.bytes, dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        # the allocating stream only (a device-wide synchronise would fail
        # while another thread's context captures its solve graph)
        torch.cuda.current_stream().synchronize()
        ftk_bind_workspace(self.handle, workspace.data_ptr(), workspace.numel())

    # thin method forms of the C calls
    def tpq_init(self, seed, sample=0, ell=0.5):
        ftk_tpq_init(self.handle, seed, sample, ell)

    def set_state(self, v, ell=0.5):
        ftk_set_state(self.handle, v, ell)

    def tpq_step(self, n_steps, save_every):
        return ftk_tpq_step(self.handle, n_steps, save_every)

    def shells(self):
        return ftk_shells(self.handle)

    def apply_op(self, shell, gamma, q, slot):
        ftk_apply_op(self.handle, shell, gamma, q, slot)

    def set_probe(self, slot, v, energy):
        ftk_set_probe(self.handle, slot, v, energy)

    def shifted_cocg(self, slots, omega, eta, tol=1e-4, max_iter=10000, allow_noconv=False):
        return ftk_shifted_cocg(self.handle, slots, omega, eta, tol, max_iter, allow_noconv)

    def spectrum(self, G, T):
        return ftk_spectrum(self.handle, G, T)

    def spectrum_ex(self, G, T, u, logQ, save_every, ell):
        return ftk_spectrum_ex(self.handle, G, T, u, logQ, save_every, ell)

    def shifted_cocg_ex(self, slots, shifts, tol=1e-4, max_iter=10000, proj_slots=None, seed_index=-1,
                        seed_switch=False, allow_noconv=False):
        return ftk_shifted_cocg_ex(self.handle, slots, shifts, tol, max_iter, proj_slots, seed_index, seed_switch,
                                   allow_noconv)

    def ctpq(self, betas, lam=1e4, first_shell=0):
        return ftk_ctpq(self.handle, betas, lam, first_shell)

    def filter_shells(self, src, e_b, eps, n_centres, n_points, tol=1e-10, max_iter=10000, first_shell=0):
        """Filtered shells with a device scratch tensor of ftk_filter_footprint
        bytes allocated (and released) here."""
        torch = self.torch
        nb = ftk_filter_footprint(n_centres, n_points, max_iter)
        if nb == 0:
            raise FtkError(FTK_EINVAL, "bad filter sizes")
        scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
        torch.cuda.current_stream().synchronize()
        try:
            return ftk_filter_shells(self.handle, src, e_b, eps, n_centres, n_points, tol, max_iter,
                                     scratch.data_ptr(), nb, first_shell)
        finally:
            self.stream.synchronize()
            del scratch

    def filter_spectrum(self, G, energy, norm2, beta, eps, T):
        return ftk_filter_spectrum(self.handle, G, energy, norm2, beta, eps, T)

    def hv(self, v, out=None):
        """v: torch tensor [dim] or [B, dim] (B vectors, one after the other)
        of complex128/complex64 on cuda; for "df" complex64 [2 B, dim] (the hi
        parts of the B vectors, then their lo parts)."""
        torch = self.torch
        n_rhs = 1 if v.dim() == 1 else v.shape[0]
        if self.prec == FTK_DF:
            n_rhs //= 2
        if out is None:
            out = torch.empty_like(v)
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        ftk_hv(self.handle, v.data_ptr(), out.data_ptr(), n_rhs)
        cur.wait_stream(self.stream)
        return out

    def get_vector(self, which):
        return ftk_get_vector(self.handle, which, self.dim)

    def autotune(self, n_rhs=1, which=0):
        return ftk_autotune(self.handle, n_rhs, which)

    def set_relax(self, theta):
        ftk_set_relax(self.handle, theta)

    def plan_info(self):
        return ftk_plan_info(self.handle)

    def launch_count(self):
        return ftk_launch_count(self.handle)

    def close(self):
        if self.handle:
            ftk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
