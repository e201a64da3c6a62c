"""The served request stream (cfneb_inputs.serve_requests / build_request):
deterministic for a seed, arrivals inside the window and in order, both
kinds present, carbon vacancy hops with odd image counts in range and
supercells that hold the relaxed 4 x 4 x 4 field, LJ requests with their
FIRE step limit, and matched endpoint shapes for every request kind."""
import numpy as np

import cfneb_inputs as ci


def test_stream_is_deterministic_and_ordered():
    a = ci.serve_requests(seed=5, rate=20.0, window=10.0)
    b = ci.serve_requests(seed=5, rate=20.0, window=10.0)
    assert a == b
    t = [s["arrival"] for s in a]
    assert t == sorted(t) and 0.0 <= t[0] and t[-1] < 10.0
    # about rate x window arrivals (Poisson: within 5 standard deviations)
    assert abs(len(a) - 200) < 5 * np.sqrt(200)


def test_request_kinds_and_parameters():
    specs = ci.serve_requests(seed=5, rate=20.0, window=30.0, img_lo=7, img_hi=16)
    kinds = {s["kind"] for s in specs}
    assert kinds == {"lj_vacancy", "tersoff_diamond_vacancy"}
    for s in specs:
        assert 7 <= s["n_images"] <= 16
        if s["kind"] == "tersoff_diamond_vacancy":
            assert s["n_images"] % 2 == 1            # one image on the saddle
            assert min(s["reps"]) >= 4                # holds the relaxed field
            assert (s["dt"], s["dt_max"], s["maxstep"]) == (0.05, 0.2, 0.1)
        else:
            assert min(s["reps"]) >= 2
            assert (s["dt"], s["dt_max"]) == (0.01, 0.03)


def test_built_requests_have_matched_endpoints():
    specs = ci.serve_requests(seed=5, rate=20.0, window=4.0)
    seen = set()
    for s in specs:
        if s["kind"] in seen:
            continue
        seen.add(s["kind"])
        (R0, h0, R1, h1), pot = ci.build_request(s)
        assert R0.shape == R1.shape and h0.shape == h1.shape == (3, 3)
        assert pot == ("lj" if s["kind"] == "lj_vacancy" else "tersoff")
        if s["kind"] == "tersoff_diamond_vacancy":
            assert len(R0) == 8 * int(np.prod(s["reps"])) - 1
    assert seen == {"lj_vacancy", "tersoff_diamond_vacancy"}
