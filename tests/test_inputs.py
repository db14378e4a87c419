"""The seeded input recipes (dp_inputs) against their stated definitions: the
counter generator against SplitMix64 written out with Python integers, and the
workload shapes, well placements, value distributions and request stream
against the recipe each docstring states."""
import math

import numpy as np

import dp_inputs as di

M64 = (1 << 64) - 1


def _splitmix64(state):
    """SplitMix64 (Steele, Lea and Flood 2014; Vigna's constants): the next
    state and output."""
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def test_counter_uniforms_are_splitmix64():
    state, outs = 0, []
    for _ in range(6):
        state, z = _splitmix64(state)
        outs.append(z)
    assert outs[0] == 0xE220A8397B1DCDAF          # the generator's first output from seed 0
    want = np.array([((z >> 11) + 0.5) / 2.0 ** 53 for z in outs])
    got = di.splitmix64_uniform(0, 0, np.arange(6))
    np.testing.assert_array_equal(got, want)
    # another (seed, stream): the same sequence started from seed*G + stream*S
    key = (5 * 0x9E3779B97F4A7C15 + 3 * 0xD1B54A32D192ED03) & M64
    state, z = _splitmix64((key + 2 * 0x9E3779B97F4A7C15) & M64)
    assert di.splitmix64_uniform(5, 3, np.array([2]))[0] == ((z >> 11) + 0.5) / 2.0 ** 53


def test_bench_field_recipe():
    prob = di.field8m()
    assert (prob.nx, prob.ny, prob.nz) == (200, 200, 50) and prob.n_cells == 4_000_000
    inj = sorted((w.i, w.j) for w in prob.wells if w.kind == di.WELL_RATE_INJ)
    prod = sorted((w.i, w.j) for w in prob.wells if w.kind == di.WELL_BHP)
    assert inj == [(a, b) for a in (50, 100, 150) for b in (50, 100, 150)]
    assert prod == [(a, b) for a in (25, 75, 125, 175) for b in (25, 75, 125, 175)]
    assert all(w.k_top == 0 and w.k_bot == 49 for w in prob.wells)
    lk = np.log(prob.kf / di.MD)
    assert abs(lk.mean() - math.log(100.0)) < 0.01 and abs(lk.std() - 2.0) < 0.01
    lm = np.log(prob.km / di.MD)
    assert abs(lm.mean() - math.log(0.05)) < 0.01 and abs(lm.std() - 0.5) < 0.01


def test_served_and_ensemble_recipes():
    sizes = [di.served_member(r).n_cells for r in range(128)]
    assert sum(sizes) == 26_766_020
    assert 9_000 <= min(sizes) and max(sizes) <= 1_100_000
    ens = [di.ensemble_member(r) for r in (0, 63)]
    assert (ens[0].nx, ens[0].nz, ens[1].nx, ens[1].nz) == (20, 5, 80, 20)
    arrivals, real, dts = di.request_stream()
    assert len(arrivals) == 512 and arrivals[0] == 0.0 and (np.diff(arrivals) > 0).all()
    rate = 511 / arrivals[-1]
    assert 170.0 < rate < 230.0                    # Poisson at 200/s
    assert set(np.unique(dts)) <= {1.0, 2.0, 5.0, 10.0} and real.max() < 128


def test_paper_examples_on_their_grids_and_at_example_3_size():
    e1, e2 = di.paper_example(1), di.paper_example(2)
    assert [(w.i, w.j) for w in e1.wells] == [(4, 0), (0, 9), (9, 9)]   # cells [5 1 1], [1 10 1], [10 10 1]
    assert [(w.i, w.j) for w in e2.wells] == [(4, 4), (0, 0), (9, 9)]
    assert (e1.nz, e2.nz) == (1, 3)
    e3 = di.paper_example(1, grid=(500, 500, 50))
    assert e3.n_cells == 25_000_000
    assert [(w.i, w.j, w.k_top, w.k_bot) for w in e3.wells] == [(225, 25, 0, 0), (25, 475, 0, 0),
                                                             (475, 475, 0, 0)]
    # the top layer's centre at 2000 ft, 100 ft layers
    assert abs((e3.top_depth + 0.5 * e3.dz) / di.FT - 2000.0) < 1e-9
