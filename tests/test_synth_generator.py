"""The seeded input generator's counter-based normals (synth.counter_normals) against their
definition: SplitMix64's published first output, a scalar big-integer evaluation of the same
definition, and the moments of N(0, 1). These are inputs, not the method; the pins make sure
that the host and device implementations draw what the definition says."""
import math

import numpy as np

import synth
from synth import lattice as lat

U64 = (1 << 64) - 1


def test_splitmix64_first_output_for_seed_zero():
    # SplitMix64 seeded with 0: its first output (Steele, Lea & Flood 2014; reference implementation).
    assert lat._sm_mix_int(lat.SM_GAMMA) == 0xE220A8397B1DCDAF


def _scalar_normal(seed, stream, t):
    key = synth.counter_key(seed, stream)
    h1 = lat._sm_mix_int((key + (2 * t + 1) * lat.SM_GAMMA) & U64) >> 11
    h2 = lat._sm_mix_int((key + (2 * t + 2) * lat.SM_GAMMA) & U64) >> 11
    u1 = (h1 + 1) * 2.0 ** -53
    u2 = h2 * (2.0 ** -53 * 2.0 * math.pi)
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(u2)


def test_vectorised_normals_match_scalar_definition():
    for seed, stream, start in ((0, 0, 0), (1000, (1 << 40) + 5, 17), (2**63 + 3, 12, 1 << 33)):
        v = synth.counter_normals(seed, stream, start, 64, chunk=7)
        ref = np.array([_scalar_normal(seed, stream, start + t) for t in range(64)])
        assert np.array_equal(v, ref)


def test_normals_moments_and_independence_of_streams():
    n = 1 << 20
    a = synth.counter_normals(5, 1, 0, n)
    b = synth.counter_normals(5, 2, 0, n)
    assert abs(a.mean()) < 5 / math.sqrt(n)
    assert abs(a.var() - 1) < 5 * math.sqrt(2 / n)
    assert abs(np.mean(a ** 4) - 3) < 0.05
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(n)
    # a block regenerates identically on its own
    assert np.array_equal(synth.counter_normals(5, 1, 1000, 10), a[1000:1010])


def test_real_space_B_recipe():
    spec = synth.CONFIGS["tiny_2x2x1"]
    B = synth.real_space_B(spec, 3, 5)
    # pair-symmetrised: B[P, mu, R1, nu, R2] = B[P, nu, R2, mu, R1]
    assert np.array_equal(B, B.transpose(0, 3, 4, 1, 2))
    w = np.exp(-spec.decay * synth.min_image_norm(spec.mesh))
    na, nk = spec.n_ao, spec.nk
    g = synth.counter_normals(spec.seed, lat._STREAM_B + 4, 0, na * nk * na * nk).reshape(na, nk, na, nk)
    g = g * w[None, :, None, None] * w[None, None, None, :]
    assert np.allclose(B[1], 0.5 * (g + g.transpose(2, 3, 0, 1)), rtol=0, atol=1e-15)
