"""The device implementation of the seeded inputs (synth.gpu) against the host one (synth/lattice.py):
the same numbers up to the last-bit rounding of log and cos."""
import numpy as np
import pytest

import synth
from synth import lattice as lat

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def test_device_normals_match_host():
    torch = torch_cuda()
    from synth import gpu
    d = gpu.counter_normals_device(torch, 1234, lat._STREAM_B + 7, 3, 5000).cpu().numpy()
    for s in range(3):
        h = synth.counter_normals(1234, lat._STREAM_B + 7 + s, 0, 5000)
        assert np.abs(d[s] - h).max() <= 1e-14 * np.abs(h).max()


@pytest.mark.parametrize("name", ["tiny_2x2x1", "hbn_4x4x1"])
def test_device_L_pairs_match_host(name):
    torch = torch_cuda()
    from synth import gpu
    import paper_1909_08596_gb300 as dm
    spec = synth.CONFIGS[name]
    if name == "hbn_4x4x1":
        spec = synth.spec_with(spec, n_aux=12)
    pairs = dm.dmet_emb_l_pairs(dm.make_desc(spec.mesh, spec.n_ao, spec.n_aux, spec.n_emb))
    d = gpu.make_L_pairs_device(torch, spec, pairs, p_block=5).cpu().numpy()
    h = synth.make_L_pairs(spec, pairs, p_block=5)
    assert np.abs(d - h).max() <= 1e-13 * np.abs(h).max()
    full = gpu.L_blocks_device(torch, spec, 2, 9).cpu().numpy()
    assert np.abs(full - synth.make_L(spec)[:, :, 2:9]).max() <= 1e-13 * np.abs(h).max()
