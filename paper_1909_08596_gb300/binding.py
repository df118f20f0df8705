"""Thin ctypes binding of libdmetemb.so (include/dmet_emb.h), same names as the C entry points.

Argument marshalling only: buffers are torch tensors (device or host) or numpy arrays
(host), passed to the library as raw pointers. Every step of the computation runs in the
library's CUDA kernels; if the library has not been built this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB
HEADER = os.path.join(_build.ROOT, "include", "dmet_emb.h")

# dmet_status_t
DMET_OK = 0
DMET_ERR_INVALID_ARG = 1
DMET_ERR_ALIGNMENT = 2
DMET_ERR_OOM = 3
DMET_ERR_NOT_ORTHONORMAL = 4
DMET_ERR_CUDA = 5
DMET_ERR_TIMEOUT = 6
DMET_ERR_UNSUPPORTED = 7
DMET_ERR_SYMMETRY = 8
STATUS_NAMES = {0: "DMET_OK", 1: "DMET_ERR_INVALID_ARG", 2: "DMET_ERR_ALIGNMENT", 3: "DMET_ERR_OOM",
                4: "DMET_ERR_NOT_ORTHONORMAL", 5: "DMET_ERR_CUDA", 6: "DMET_ERR_TIMEOUT",
                7: "DMET_ERR_UNSUPPORTED", 8: "DMET_ERR_SYMMETRY"}
# dmet_prec_t, dmet_sym_t, dmet_pack_t
DMET_PREC_FP64, DMET_PREC_BF16X3, DMET_PREC_TF32, DMET_PREC_TF32X3, DMET_PREC_FP16X2 = 0, 1, 2, 3, 4
DMET_SYM_NONE, DMET_SYM_REAL = 0, 1
DMET_PACK_AUTO, DMET_PACK_S8, DMET_PACK_FULL, DMET_PACK_S4 = 0, 1, 2, 3
# dmet_l_layout_t
DMET_L_FULL, DMET_L_REDUCED = 0, 1


class DmetError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class dmet_emb_desc_t(ctypes.Structure):
    _fields_ = [
        ("mesh", ctypes.c_int32 * 3),
        ("n_ao", ctypes.c_int32),
        ("n_aux", ctypes.c_int32),
        ("n_spin", ctypes.c_int32),
        ("n_emb", ctypes.c_int32 * 2),
        ("prec", ctypes.c_int32),
        ("ck_norm", ctypes.c_int32),
        ("sym", ctypes.c_int32),
        ("eri_pack", ctypes.c_int32),
        ("check_l", ctypes.c_int32),
        ("l_layout", ctypes.c_int32),
        ("q_begin", ctypes.c_int32),
        ("q_end", ctypes.c_int32),
        ("ortho_tol", ctypes.c_double),
        ("sym_tol", ctypes.c_double),
    ]


def make_desc(mesh, n_ao, n_aux, n_emb, n_spin=1, prec=DMET_PREC_FP64, ck_norm=0, sym=DMET_SYM_REAL,
              eri_pack=DMET_PACK_AUTO, check_l=0, ortho_tol=0.0, sym_tol=0.0, l_layout=0, q_range=None
              ) -> dmet_emb_desc_t:
    d = dmet_emb_desc_t()
    d.mesh[:] = list(mesh)
    d.n_ao, d.n_aux, d.n_spin = n_ao, n_aux, n_spin
    ne = list(n_emb) if isinstance(n_emb, (list, tuple)) else [n_emb, n_emb if n_spin == 2 else 0]
    d.n_emb[:] = ne + [0] * (2 - len(ne))
    d.prec, d.ck_norm, d.sym, d.eri_pack, d.check_l = prec, ck_norm, sym, eri_pack, check_l
    d.l_layout = l_layout
    d.q_begin, d.q_end = (0, 0) if q_range is None else (int(q_range[0]), int(q_range[1]))
    d.ortho_tol, d.sym_tol = ortho_tol, sym_tol
    return d


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1909_08596_gb300.build.build() "
                               "(or __graft_entry__.build()); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        L.dmet_emb_eri_bytes.argtypes = [ctypes.POINTER(dmet_emb_desc_t), ctypes.c_int32]
        L.dmet_emb_eri_bytes.restype = ctypes.c_size_t
        L.dmet_emb_plan.argtypes = [ctypes.POINTER(dmet_emb_desc_t), ctypes.c_int32, _P, ctypes.c_size_t,
                                    ctypes.POINTER(_P)]
        L.dmet_emb_plan.restype = st
        L.dmet_emb_transform_3idx.argtypes = [_P, ctypes.c_int32, _P, ctypes.POINTER(_P), ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(_P)]
        L.dmet_emb_transform_3idx.restype = st
        L.dmet_emb_eri.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.POINTER(_P)),
                                   ctypes.POINTER(ctypes.POINTER(_P))]
        L.dmet_emb_eri.restype = st
        L.dmet_emb_status.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        L.dmet_emb_status.restype = st
        L.dmet_emb_destroy.argtypes = [_P]
        L.dmet_emb_destroy.restype = st
        ip = ctypes.POINTER(ctypes.c_int32)
        L.dmet_emb_schedule.argtypes = [ctypes.POINTER(dmet_emb_desc_t), ip, ip, ip, ip, ip, ip]
        L.dmet_emb_schedule.restype = st
        L.dmet_emb_l_pairs.argtypes = [ctypes.POINTER(dmet_emb_desc_t), ip, ctypes.POINTER(ctypes.c_int64)]
        L.dmet_emb_l_pairs.restype = st
        L.dmet_emb_profile.argtypes = [_P, ctypes.c_int32]
        L.dmet_emb_profile.restype = st
        L.dmet_emb_fock.argtypes = [_P, ctypes.c_int32, _P, _P, _P, _P, _P]
        L.dmet_emb_fock.restype = st
        L.dmet_emb_bath.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.POINTER(ctypes.c_int32),
                                    ctypes.c_int32, _P, _P]
        L.dmet_emb_bath.restype = st
        L.dmet_emb_jk_df.argtypes = [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]
        L.dmet_emb_jk_df.restype = st
        L.dmet_emb_eri_fftdf.argtypes = [_P, ctypes.c_int32, _P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_P)]
        L.dmet_emb_eri_fftdf.restype = st
        L.dmet_fftdf_plane_waves.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                                             _P, _P, _P]
        L.dmet_fftdf_plane_waves.restype = st
        L.dmet_emb_profile_count.argtypes = []
        L.dmet_emb_profile_count.restype = ctypes.c_int32
        L.dmet_emb_profile_read.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_char_p),
                                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]
        L.dmet_emb_profile_read.restype = st
        L.dmet_emb_graph.argtypes = [_P, ctypes.c_int32]
        L.dmet_emb_graph.restype = st
        L.dmet_emb_batch_mode.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.dmet_emb_batch_mode.restype = st
        L.dmet_emb_split_parts.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.dmet_emb_split_parts.restype = st
        L.dmet_emb_problem_ms.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        L.dmet_emb_problem_ms.restype = st
        L.dmet_emb_autotune.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.POINTER(_P)),
                                        ctypes.POINTER(ctypes.POINTER(_P))]
        L.dmet_emb_autotune.restype = st
        L.dmet_emb_tile_widths.argtypes = [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
        L.dmet_emb_tile_widths.restype = st
        L.dmet_emb_wait_limit.argtypes = [_P, ctypes.c_uint64, ctypes.c_int32]
        L.dmet_emb_wait_limit.restype = st
        L.dmet_emb_launch_count.argtypes = [_P]
        L.dmet_emb_launch_count.restype = ctypes.c_int64
        L.dmet_emb_eri_noalloc.argtypes = [ctypes.POINTER(dmet_emb_desc_t), _P, ctypes.POINTER(_P),
                                           ctypes.POINTER(_P), _P]
        L.dmet_emb_eri_noalloc.restype = st
        L.dmet_emb_last_error.argtypes = []
        L.dmet_emb_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def declared_symbols():
    """Entry points declared in include/dmet_emb.h."""
    with open(HEADER) as f:
        src = f.read()
    return sorted(set(re.findall(r"DMET_API\s+[\w\s\*]+?\b(dmet_emb_\w+)\s*\(", src)))


def _check(status):
    if status != DMET_OK:
        raise DmetError(status, lib().dmet_emb_last_error().decode())


def ptr(buf) -> int:
    """Raw address of a contiguous torch tensor or numpy array (None -> 0)."""
    if buf is None:
        return 0
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("numpy buffer must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    if isinstance(buf, int):
        return buf
    raise TypeError(f"unsupported buffer type {type(buf)}")


def _descs(descs):
    if isinstance(descs, dmet_emb_desc_t):
        descs = [descs]
    arr = (dmet_emb_desc_t * len(descs))(*descs)
    return arr, len(descs)


def dmet_emb_eri_bytes(desc, block):
    return int(lib().dmet_emb_eri_bytes(ctypes.byref(desc), block))


def dmet_emb_plan(descs, stream=None, workspace_limit=0):
    """Plan handle (int) for a desc or list of descs; `stream` is a cudaStream_t value."""
    arr, n = _descs(descs)
    out = _P()
    _check(lib().dmet_emb_plan(arr, n, _P(stream or 0), workspace_limit, ctypes.byref(out)))
    return out.value


def dmet_emb_transform_3idx(plan, problem, L, C, q_begin, q_end, Lq_out):
    cs = (_P * len(C))(*[ptr(c) for c in C])
    outs = (_P * len(Lq_out))(*[ptr(o) for o in Lq_out])
    _check(lib().dmet_emb_transform_3idx(_P(plan), problem, _P(ptr(L)), cs, q_begin, q_end, outs))


def _problem_arrays(L, C, eri_out):
    n = len(L)
    ls = (_P * n)(*[ptr(x) for x in L])
    crows = [(_P * len(c))(*[ptr(x) for x in c]) for c in C]
    erows = [(_P * len(e))(*[ptr(x) for x in e]) for e in eri_out]
    cp = (ctypes.POINTER(_P) * n)(*[ctypes.cast(r, ctypes.POINTER(_P)) for r in crows])
    ep = (ctypes.POINTER(_P) * n)(*[ctypes.cast(r, ctypes.POINTER(_P)) for r in erows])
    return ls, cp, ep, (crows, erows)


def dmet_emb_eri(plan, L, C, eri_out):
    """L: list over problems; C: list over problems of lists over spins; eri_out: list of lists."""
    ls, cp, ep, _keep = _problem_arrays(L, C, eri_out)
    _check(lib().dmet_emb_eri(_P(plan), ls, cp, ep))


def dmet_emb_autotune(plan, L, C, eri_out):
    ls, cp, ep, _keep = _problem_arrays(L, C, eri_out)
    _check(lib().dmet_emb_autotune(_P(plan), ls, cp, ep))


def dmet_emb_tile_widths(plan, problem):
    bn = (ctypes.c_int32 * 2)()
    _check(lib().dmet_emb_tile_widths(_P(plan), problem, bn))
    return list(bn)


def dmet_emb_eri_noalloc(desc, L, C, eri_out, stream=None):
    """One problem's FP64 8-fold packed ERIs with no allocation (device buffers only)."""
    cs = (_P * len(C))(*[ptr(c) for c in C])
    outs = (_P * len(eri_out))(*[ptr(o) for o in eri_out])
    _check(lib().dmet_emb_eri_noalloc(ctypes.byref(desc), _P(ptr(L)), cs, outs, _P(stream or 0)))


def dmet_emb_status(plan, problem, raise_on_error=False):
    """(status, stats[4]) after waiting for the plan's stream."""
    stats = (ctypes.c_double * 4)()
    s = lib().dmet_emb_status(_P(plan), problem, stats)
    if raise_on_error:
        _check(s)
    return s, list(stats)


def dmet_emb_destroy(plan):
    _check(lib().dmet_emb_destroy(_P(plan)))


def dmet_emb_schedule(desc):
    nk = int(np.prod(list(desc.mesh)))
    a = {k: np.zeros(nk * nk if k in ("k2_of", "rep_k1", "rep_half") else nk, dtype=np.int32)
         for k in ("k2_of", "neg", "q_weight", "n_rep", "rep_k1", "rep_half")}
    ip = ctypes.POINTER(ctypes.c_int32)
    args = [a[k].ctypes.data_as(ip) for k in ("k2_of", "neg", "q_weight", "n_rep", "rep_k1", "rep_half")]
    _check(lib().dmet_emb_schedule(ctypes.byref(desc), *args))
    a["k2_of"] = a["k2_of"].reshape(nk, nk)
    a["rep_k1"] = a["rep_k1"].reshape(nk, nk)
    a["rep_half"] = a["rep_half"].reshape(nk, nk)
    return a


def dmet_emb_l_pairs(desc):
    """The (k1 Nk + k2) blocks of the reduced L layout, in its order (int32 array)."""
    n = ctypes.c_int64()
    _check(lib().dmet_emb_l_pairs(ctypes.byref(desc), None, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.int32)
    _check(lib().dmet_emb_l_pairs(ctypes.byref(desc), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  ctypes.byref(n)))
    return out


def dmet_emb_profile(plan, enable):
    _check(lib().dmet_emb_profile(_P(plan), 1 if enable else 0))


def dmet_emb_fock(plan, F, C, eri, gamma, fock_out, problem=0):
    """Embedding Fock matrix with the double counting removed (device tensors; see dmet_emb_fock)."""
    _check(lib().dmet_emb_fock(_P(plan), problem, ptr(F), ptr(C), ptr(eri), ptr(gamma), ptr(fock_out)))


def dmet_emb_bath(plan, gamma_k, C_lo, val, C_out, info=None, problem=0, spin=0):
    """DMET bath and embedding orbitals C^{k,AO,EO} on the device (see dmet_emb_bath)."""
    v = (ctypes.c_int32 * len(val))(*[int(x) for x in val])
    _check(lib().dmet_emb_bath(_P(plan), problem, spin, ptr(gamma_k), ptr(C_lo), v, len(val), ptr(C_out),
                               ptr(info) if info is not None else None))


def dmet_emb_jk_df(plan, Lq, gamma, J, K, problem=0, spin=0):
    """Density-fitted Coulomb and exchange of gamma from the factors L^q (device tensors; see dmet_emb_jk_df)."""
    _check(lib().dmet_emb_jk_df(_P(plan), problem, spin, ptr(Lq), ptr(gamma), ptr(J), ptr(K)))


def dmet_emb_eri_fftdf(plan, rho, C, grid, lattice, eri_out, problem=0):
    """FFTDF embedded ERIs (Algorithm 2) from pair densities rho [Nk][Nk][N_g][n_ao][n_ao] (device tensors)."""
    cs = (_P * len(C))(*[ptr(c) for c in C])
    outs = (_P * len(eri_out))(*[ptr(o) for o in eri_out])
    gr = (ctypes.c_int32 * 3)(*[int(x) for x in grid])
    la = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()])
    _check(lib().dmet_emb_eri_fftdf(_P(plan), problem, _P(ptr(rho)), cs, gr, la, outs))


def dmet_fftdf_plane_waves(mesh, q, grid, lattice):
    """(m [N_g, 3] int32, v [N_g] float64, opposite [N_g] int32) of the FFTDF plane waves at momentum q
    (host-only; see dmet_fftdf_plane_waves)."""
    ng = int(np.prod(grid))
    m = np.zeros((ng, 3), dtype=np.int32)
    v = np.zeros(ng, dtype=np.float64)
    opp = np.zeros(ng, dtype=np.int32)
    me = (ctypes.c_int32 * 3)(*[int(x) for x in mesh])
    gr = (ctypes.c_int32 * 3)(*[int(x) for x in grid])
    la = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(lattice, dtype=np.float64).ravel()])
    _check(lib().dmet_fftdf_plane_waves(me, int(q), gr, la, ptr(m), ptr(v), ptr(opp)))
    return m, v, opp


def dmet_emb_profile_count():
    return int(lib().dmet_emb_profile_count())


def dmet_emb_profile_read(plan, kernel):
    name = ctypes.c_char_p()
    launches = ctypes.c_int64()
    ms, fl, ex, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().dmet_emb_profile_read(_P(plan), kernel, ctypes.byref(name), ctypes.byref(launches),
                                       ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(ex), ctypes.byref(by)))
    return {"name": name.value.decode(), "launches": launches.value, "ms": ms.value, "flops": fl.value,
            "exec_flops": ex.value, "bytes": by.value}


def dmet_emb_graph(plan, enable):
    _check(lib().dmet_emb_graph(_P(plan), 1 if enable else 0))


def dmet_emb_batch_mode(plan, mode):
    """Sets the batch mode (1 grouped launches, 0 per-problem side streams); returns whether calls
    with device buffers will run grouped."""
    active = ctypes.c_int32()
    _check(lib().dmet_emb_batch_mode(_P(plan), int(mode), ctypes.byref(active)))
    return bool(active.value)


def dmet_emb_split_parts(plan, problem):
    """[(tiles split, parts per tile)] of the aa, ab and bb contraction blocks."""
    a = (ctypes.c_int32 * 6)()
    _check(lib().dmet_emb_split_parts(_P(plan), problem, a))
    return [(a[2 * b], a[2 * b + 1]) for b in range(3)]


def dmet_emb_problem_ms(plan, problem):
    ms = ctypes.c_double()
    _check(lib().dmet_emb_problem_ms(_P(plan), problem, ctypes.byref(ms)))
    return ms.value


def dmet_emb_wait_limit(plan, wait_ns, test_withhold_loads=False):
    _check(lib().dmet_emb_wait_limit(_P(plan), int(wait_ns), 1 if test_withhold_loads else 0))


def dmet_emb_launch_count(plan):
    return int(lib().dmet_emb_launch_count(_P(plan)))


def dmet_emb_last_error():
    return lib().dmet_emb_last_error().decode()
