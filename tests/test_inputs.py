"""The seeded generator: SplitMix64 reference values and distribution sanity."""
import numpy as np

import fc_inputs


def test_splitmix64_reference_values():
    # First outputs of SplitMix64 seeded with 0 and 1234567 (Vigna's reference C
    # implementation, next() called repeatedly from the given state).
    assert [int(v) for v in fc_inputs.splitmix64(0, 0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in fc_inputs.splitmix64(1234567, 0, 2)] == [
        6457827717110365317, 3203168211198807973]


def test_problem_layout_and_ranges():
    p = fc_inputs.problem(32, seed=0, with_t=True)
    assert p["s"].shape == (1024,) and np.all((p["s"] > 0.5) & (p["s"] < 1.5))
    assert np.all(p["b"] == 1.0)
    assert np.all((p["t"] > 0) & (p["t"] < 1))
    q = fc_inputs.problem(32, seed=0, with_t=True)
    assert np.array_equal(p["s"], q["s"]) and np.array_equal(p["t"], q["t"])
    r = fc_inputs.problem(32, seed=1)
    assert not np.array_equal(p["s"], r["s"])


def test_normal_moments():
    v, used = fc_inputs.normal(7, 0, 200001)
    assert used == 200002
    assert abs(v.mean()) < 0.01 and abs(v.std() - 1) < 0.01


def test_request_stream():
    reqs = fc_inputs.request_stream(2000, seed=3, rate_per_s=100.0)
    Ls = np.array([r["L"] for r in reqs])
    assert set(Ls) <= {32, 64, 128, 256, 512, 1024, 2048}
    # endpoints have half weight under rounding of the log-uniform exponent
    assert (Ls == 32).mean() < (Ls == 256).mean()
    t = np.array([r["arrival_s"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.01) < 0.001
