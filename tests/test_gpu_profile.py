"""The launch-timing API (tt_profile_*) that the bench reads its per-kernel
times from: one (pack, forward, adjoint) triple per gradient evaluation, times
that add up to no more than the stream time around them, and events recycled
over more launches than the handle pre-creates."""
import pytest
import torch

from paper_2504_16446_gb300 import synth, tt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2504_16446_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_profile_counts_and_times_every_launch():
    st = synth.small_setup(n=(12, 9, 10), nj=13, nk=11, ell_max=4, n_proj=9, n_seg=5, seed=1)
    h = tt.Handle(st, "f32")
    c = torch.as_tensor(synth.random_volume(st, 3), dtype=torch.float32, device="cuda")
    I = torch.as_tensor(synth.random_data(st, 4), dtype=torch.float32, device="cuda")
    g = torch.empty_like(c)
    h.gradient_residual(c, I, out=g)
    n = 300                        # 900 launches, 1800 events: well past the pre-created pool
    h.profile(True)
    h.profile_reset()
    launches0 = h.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    losses = [h.gradient_residual(c, I, out=g)[0] for _ in range(n)]
    e1.record()
    torch.cuda.synchronize()
    p = h.profile_read()
    h.profile(False)
    assert h.launch_count() - launches0 == 3 * n
    for k in ("pack", "forward", "adjoint"):
        assert p[k][1] == n, (k, p[k])
        assert p[k][0] > 0
    assert sum(v[0] for v in p.values()) <= e0.elapsed_time(e1)
    assert len(set(losses)) == 1   # profiling changes nothing in the result
    # a read without new launches returns the same totals; a reset clears them
    assert h.profile_read() == p
    h.profile_reset()
    assert all(v == (0.0, 0) for v in h.profile_read().values())
    h.close()


def test_profile_chain_over_several_adjoint_launches():
    """300 projections: the adjoint runs as two launches (256 projections per
    parameter block), all four launches of an evaluation sharing boundary
    events; every launch is still counted and timed, and the results are
    those of an unprofiled evaluation."""
    st = synth.small_setup(n=(7, 6, 9), nj=8, nk=7, ell_max=4, n_proj=300, n_seg=5, seed=41)
    h = tt.Handle(st, "f32")
    c = torch.as_tensor(synth.random_volume(st, 42), dtype=torch.float32, device="cuda")
    I = torch.as_tensor(synth.random_data(st, 43), dtype=torch.float32, device="cuda")
    loss0, g0 = h.gradient_residual(c, I)
    h.profile(True)
    h.profile_reset()
    for _ in range(50):
        loss, g = h.gradient_residual(c, I)
    p = h.profile_read()
    h.profile(False)
    assert p["pack"][1] == 50 and p["forward"][1] == 50 and p["adjoint"][1] == 100
    assert all(p[k][0] > 0 for k in ("pack", "forward", "adjoint"))
    assert loss == loss0
    torch.testing.assert_close(g, g0, rtol=0, atol=0)
    h.close()
