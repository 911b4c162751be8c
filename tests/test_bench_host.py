"""Host-side arithmetic of bench.py (no GPU): slab counts of a partition and
the error definitions of the time-to-1 % metric."""
import numpy as np

import bench


def test_subdomain_slabs():
    # 8 slabs in 2 parts, overlap 1: parts [0,4) -> [0,5), [4,8) -> [3,8)
    fwd, bwd = bench._subdomain_slabs(8, [0, 4, 8], [1, 1])
    assert fwd == 5 + 5
    # backward: part 0 from slab 3 down to 0 (lo = 0): 4; part 1 (lo = 1): from 3 down to 0 -> 4
    assert bwd == 4 + 4
    # one part: n_t forward, n_t - 1 backward
    assert bench._subdomain_slabs(8, [0, 8], [0]) == (8, 7)


def test_seed_errors_definition():
    v_ex = np.array([1.0, 2.0, 4.0])
    t_ex = np.array([1.0, -2.0, 10.0])
    vs = [v_ex * 1.01, v_ex * 0.99]
    gs = [t_ex * 1.02, t_ex * 0.98]
    e = bench._seed_errors(vs, gs, v_ex, t_ex)
    assert abs(e["eps_diag"] - 0.01) < 1e-12
    assert all(abs(x - 0.02) < 1e-12 for x in e["eps_traces"])
    assert e["seeds"] == 2 and not e["meets_1pct"]


def test_oracle_sample_exact_form_and_half_blocks():
    """The CPU baseline's sample: the exact one-part form extrapolates the
    2-slab chain to n_t slabs, plain RBMC to its parts' slabs plus the direct
    sampler; the half-block sample takes the leading half of every block and
    states its cubic scaling."""
    import qsel_inputs as qi
    w = qi.workload("grid16_nt8")
    est_ex, spent, desc = bench.oracle_sample(w)
    assert est_ex > 0 and spent > 0 and f"the {w.n_t} slabs of the exact one-part" in desc
    est_rb, _, desc_rb = bench.oracle_sample(w, exact=False)
    assert "plain RBMC" in desc_rb and est_rb > 0
    est_h, _, desc_h = bench.oracle_sample(w, frac=0.5)
    assert est_h > 0 and "leading 128x128 of every block" in desc_h and "x 8.0" in desc_h
