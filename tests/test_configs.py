"""The seeded synthetic workloads (host logic, no GPU): reproducible from the
seed, inside the stated ranges, and built by the stated rules."""
import numpy as np

from paper_1705_06807_gb300 import configs as K


def test_batch_instances_are_seeded_and_in_range():
    a, b = K.batch_instances(256, seed=0), K.batch_instances(256, seed=0)
    assert a == b and a != K.batch_instances(256, seed=1)
    Rs = np.array([q["n_replicas"] for q in a])
    assert Rs.min() >= 64 and Rs.max() <= 65536
    assert 2.0e6 < Rs.sum() < 3.0e6  # log-uniform mean about 9.4e3 per instance
    for i, q in enumerate(a):
        net = q["network"]
        if i % 2 == 0:
            V = net["s"][2]
            assert net["kind"] == "schlogl" and V in (0.5, 1.0, 2.0, 4.0, 8.0)
            assert q["x0"] == [int(round(85 * V))] and net["regions"][0][1] == int(round(250 * V))
        else:
            alpha, hill = net["c"][0], net["c"][1]
            assert net["kind"] == "toggle" and 30.0 <= alpha <= 80.0 and 2.0 <= hill <= 3.0
            hm = net["hist_max"][0]
            assert hm == max(63, int(np.ceil(alpha + 10.0 * np.sqrt(alpha) + 20.0))) and q["x0"] == [int(alpha), 0]


def test_serve_requests_are_a_seeded_poisson_stream():
    s = K.serve_requests(rate=200.0, seconds=20.0, seed=0)
    assert s == K.serve_requests(rate=200.0, seconds=20.0, seed=0)
    t = np.array([a for a, _ in s])
    assert np.all(np.diff(t) > 0) and t[-1] < 20.0
    assert abs(len(s) - 4000) < 4.5 * np.sqrt(4000)  # Poisson count with mean rate * seconds
    T = np.array([q["T_end"] for _, q in s])
    assert T.min() >= 1e3 and T.max() <= 1e5
    kinds = [q["network"]["kind"] for _, q in s]
    assert abs(kinds.count("toggle") / len(kinds) - 0.5) < 0.05


def test_genetic_switch_spec_carries_the_paper_constants():
    g = K.genetic_switch()
    b = 22.5
    assert g["c"] == [2400.0 / b, b, 50.0, 24.0 / b, 2400.0 / b, 24.0 / b, 2400.0 / b, 1000.0]
    assert g["hist_max"] == [31, 3500] and g["regions"] == [([0, 1], 512)]
