"""Device implementation of the seeded inputs whose L is too large to draw on the host.

Same definitions as synth/lattice.py (real_space_B and fourier_L, drawn P-block by P-block):
the N(0,1) numbers come from libsynthgen.so (synth/csrc/gen.cu, the device twin of
counter_normals) and the decay, pair symmetrisation and Fourier transform are torch operations
on the device. Nothing here is the embedded-ERI method's arithmetic; the library under test
never calls this module, and its results are checked against synth/lattice.py's host
implementation on small problems (tests/test_gpu_synth.py).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build
from .lattice import _STREAM_B, LatticeSpec, min_image_norm

_lib = None


def lib():
    global _lib
    if _lib is None:
        _build.build()
        L = ctypes.CDLL(_build.LIB)
        L.synth_counter_normals.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_longlong,
                                            ctypes.c_longlong, ctypes.c_void_p]
        L.synth_counter_normals.restype = ctypes.c_int
        _lib = L
    return _lib


def counter_normals_device(torch, seed: int, stream0: int, n_streams: int, per: int):
    """[n_streams, per] float64 on the current device: normals 0 .. per-1 of streams stream0 + s."""
    out = torch.empty((n_streams, per), dtype=torch.float64, device="cuda")
    st = lib().synth_counter_normals(ctypes.c_void_p(out.data_ptr()), int(seed) & (2**64 - 1), int(stream0),
                                     int(n_streams), int(per), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise RuntimeError(f"synth_counter_normals failed with CUDA error {st}")
    return out


def real_space_B_device(torch, spec: LatticeSpec, p_begin: int, p_end: int):
    """B[P, mu, R1, nu, R2] for P in [p_begin, p_end) on the device (real_space_B's definition)."""
    nk, na = spec.nk, spec.n_ao
    w = torch.from_numpy(np.exp(-spec.decay * min_image_norm(spec.mesh))).cuda()
    g = counter_normals_device(torch, spec.seed, _STREAM_B + p_begin, p_end - p_begin, na * nk * na * nk)
    g = g.view(p_end - p_begin, na, nk, na, nk)
    g *= w.view(1, 1, nk, 1, 1)
    g *= w.view(1, 1, 1, 1, nk)
    return 0.5 * (g + g.permute(0, 3, 4, 1, 2))


def fourier_L_device(torch, Bblk, mesh):
    """L[k1, k2, P, mu, nu] = sum_{R1,R2} exp(-i k1.R1 + i k2.R2) B[P, mu, R1, nu, R2] (fourier_L's
    definition: the forward DFT over R1 and the unscaled inverse DFT over R2)."""
    npb, na, nk = Bblk.shape[0], Bblk.shape[1], Bblk.shape[2]
    n1, n2, n3 = mesh
    x = Bblk.reshape(npb, na, n1, n2, n3, na, n1, n2, n3)
    x = torch.fft.fftn(x, dim=(2, 3, 4))
    x = torch.fft.ifftn(x, dim=(6, 7, 8), norm="forward")
    return x.reshape(npb, na, nk, na, nk).permute(2, 4, 0, 1, 3)   # [k1][k2][P][mu][nu] (a view)


def make_L_pairs_device(torch, spec: LatticeSpec, pairs, out=None, p_block: int = 4):
    """L[e][P][mu][nu] = L^{k1_e, k2_e} for the listed pairs (k1 Nk + k2), complex128 on the device,
    generated P-block by P-block (make_L_pairs' definition)."""
    nk, na = spec.nk, spec.n_ao
    pairs = torch.as_tensor(np.asarray(pairs, dtype=np.int64), device="cuda")
    if out is None:
        out = torch.empty((len(pairs), spec.n_aux, na, na), dtype=torch.complex128, device="cuda")
    k1, k2 = pairs // nk, pairs % nk
    for p0 in range(0, spec.n_aux, p_block):
        p1 = min(spec.n_aux, p0 + p_block)
        x = fourier_L_device(torch, real_space_B_device(torch, spec, p0, p1), spec.mesh)
        out[:, p0:p1] = x[k1, k2]
        del x
    return out


def L_blocks_device(torch, spec: LatticeSpec, p_begin: int, p_end: int):
    """The full L[k1][k2][P][mu][nu] of aux functions [p_begin, p_end), contiguous, on the device."""
    return fourier_L_device(torch, real_space_B_device(torch, spec, p_begin, p_end), spec.mesh).contiguous()
