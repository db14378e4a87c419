"""The allocation-free residual-norm entry point against sim_get_norms.

Callers that must not allocate device memory (a serving loop that keeps an
exact device-memory budget and cannot take the device-wide synchronisation
of cudaMalloc/cudaFree, or a host whose device memory belongs to another
framework's pool) get the scaled residual norms from
dp_residual_norms_noalloc, whose scratch is a static device array.  This
file runs last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

import dp_inputs as di


@pytest.mark.gpu
@pytest.mark.parametrize("make", [di.tiny, lambda: di.layered(40, 30, 6)])
def test_noalloc_norms_match_sim_get_norms_twice(make):
    import torch
    from paper_1808_04338_gb300 import dpsim
    torch.cuda.set_device(0)
    prob = make()
    sim = dpsim.Sim(prob, dpsim.options("report"))
    rng = np.random.default_rng(11)
    sim.set_iterate(prob.p0 + rng.uniform(-2e5, 2e5, prob.n_cells),
                    rng.uniform(0.25, 0.75, prob.n_cells), prob.bhp0)
    sim.assemble(prob.dt)
    expect = sim.norms()[:2]
    _, _, _, res = sim.jacobian()
    dev = torch.device("cuda", 0)
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    kinds = t([w.kind for w in prob.wells], torch.int32)
    targets = t([w.target for w in prob.wells])
    args = (t(prob.phi_f), t(prob.phi_m), kinds, targets, t(res))
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        rc, msg = dpsim.residual_norms_noalloc(prob, *args, prob.dt, out, stream)
        assert rc == 0, msg
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the two paths scale by a division and by a product with a
        # precomputed reciprocal: entries may differ in the last bit
        np.testing.assert_allclose(got[0], expect[0], rtol=1e-12)
        np.testing.assert_allclose(got[1], expect[1], rtol=1e-15)
    sim.close()


@pytest.mark.gpu
def test_noalloc_rejects_problems_beyond_its_scratch():
    """More block rows than the static scratch covers: rejected before any
    device work, with a message naming the limit."""
    import torch
    from paper_1808_04338_gb300 import dpsim
    prob = di.tiny()
    prob.nx, prob.ny, prob.nz = 1000, 1000, 10
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    kinds = torch.zeros(2, dtype=torch.int32, device="cuda")
    rc, msg = dpsim.residual_norms_noalloc(prob, dummy, dummy, kinds, dummy, dummy, 1.0, dummy)
    assert rc == dpsim.DP_EINVAL and "static scratch limit" in msg
