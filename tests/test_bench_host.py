"""Host-side pieces of bench.py: its closed-form schedule counts (used to count useful flops without
the library, so the reference arm never loads it) against the library's schedule, and the packed
positions it compares with the oracle."""
import numpy as np
import pytest

import bench
import oracle
import paper_1909_08596_gb300 as dm


@pytest.mark.parametrize("mesh", [(1, 1, 1), (2, 1, 1), (3, 1, 1), (2, 2, 1), (3, 3, 1), (2, 2, 2), (4, 4, 4),
                                  (6, 6, 1), (3, 3, 3), (5, 1, 2)])
def test_schedule_counts_match_library(mesh):
    qw, nrep = bench.schedule_counts(mesh)
    s = dm.dmet_emb_schedule(dm.make_desc(mesh, 2, 3, 1))
    assert qw == s["q_weight"].tolist()
    assert nrep == s["n_rep"].tolist()


def test_reduced_pair_count_of_nio_shape():
    # 8 self-conjugate q with 36 orbit representatives each, 28 q < -q with 32 each
    qw, nrep = bench.schedule_counts((4, 4, 4))
    assert sum(r for w, r in zip(qw, nrep) if w) == 1184
    assert len(dm.dmet_emb_l_pairs(dm.make_desc((4, 4, 4), 104, 900, 300, n_spin=2))) == 1184


def test_block_positions_match_pair_matrix():
    import synth
    spec = synth.spec_with(synth.CONFIGS["tiny_2x2x1"], n_spin=2, n_emb=6)
    rng = np.random.default_rng(3)
    ea = rng.standard_normal((6, 6, 6, 6))
    ea = ea + ea.transpose(1, 0, 2, 3)
    ea = ea + ea.transpose(0, 1, 3, 2)
    eb = ea + ea.transpose(2, 3, 0, 1)  # 8-fold symmetric
    S = [np.array([0, 2, 5]), np.array([1, 4, 5])]
    pos = bench.block_positions(spec, S)
    packed = oracle.pack_s8(eb)
    sub = eb[np.ix_(S[0], S[0], S[0], S[0])].ravel()
    assert np.array_equal(packed[pos[0]], sub)
    ab = oracle.pair_matrix(ea).ravel()   # [IJ][KL] over alpha pairs x beta pairs
    assert np.array_equal(ab[pos[1]], ea[np.ix_(S[0], S[0], S[1], S[1])].ravel())


def test_useful_flops_nio_shape():
    import synth
    spec = synth.CONFIGS["nio_4x4x4_uhf"]
    tot, t, c = bench.useful_flops(spec, [300, 300])
    assert abs(c - 470e12) / 470e12 < 0.01      # aa + bb SYRK and the ab GEMM at K = 57 600
    assert 150e12 < t < 250e12


def test_resident_groups_cover_in_order_within_budget():
    needs = [5, 3, 9, 1, 1, 12, 2, 2]
    groups = bench.resident_groups(needs, 10)
    assert [i for g in groups for i in g] == list(range(len(needs)))
    for g in groups:
        assert len(g) == 1 or sum(needs[i] for i in g) <= 10
    assert groups == [[0, 1], [2, 3], [4], [5], [6, 7]]
    assert bench.resident_groups([], 10) == []


def test_stated_batch_specs_follow_the_stated_ranges():
    import synth
    specs = synth.batch_specs(48, n_ao_range=(26, 104), n_emb_range=(40, 300))
    assert len(specs) == 48
    assert all(26 <= s.n_ao <= 104 and 40 <= s.n_emb <= 300 for s in specs)
    assert all(s.n_aux == int(8.5 * s.n_ao + 0.5) for s in specs)
    assert {s.nk for s in specs} <= {8, 27, 36, 64}
    assert sum(s.n_spin == 2 for s in specs) == 24


def test_traffic_only_for_the_captured_kernel_sources(monkeypatch):
    key = ("w", "bf16x3", "tc_contract")
    monkeypatch.setattr(bench, "TRAFFIC", {key: (123.0, bench.kernel_sources_digest())})
    assert bench.traffic_of(key) == 123.0
    monkeypatch.setattr(bench, "TRAFFIC", {key: (123.0, "0" * 16)})
    assert bench.traffic_of(key) is None
    assert bench.traffic_of(("other", "bf16x3", "tc_contract")) is None


def test_roofline_peak_choice():
    """A step of a second or more takes the sustained bf16 peak, a short one the burst peak; the
    executed-flop fraction against the burst peak is reported beside it."""
    import synth
    spec = synth.CONFIGS["tiny_2x2x1"]
    ks = [{"name": "tc_contract", "ms": 10.0, "launches": 2, "flops": 1e12, "exec_flops": 6e12, "bytes": 1e9},
          {"name": "split_operands", "ms": 1.0, "launches": 1, "flops": 0.0, "exec_flops": 0.0, "bytes": 1e9}]
    peaks, _ = bench.measured_peaks()
    burst = bench.roofline(spec, "bf16x3", ks)
    sus = bench.roofline(spec, "bf16x3", ks, sustained=True)
    assert burst["kernel"] == sus["kernel"] == "tc_contract"
    assert burst["achieved"] == sus["achieved"] == 6e12 / 2 / (5e-3) / 1e12
    assert burst["peak"] == peaks["bf16_tflops"] and sus["peak"] == peaks["bf16_tflops_sustained"]
    assert sus["frac_of_burst_peak"] == burst["frac"]
