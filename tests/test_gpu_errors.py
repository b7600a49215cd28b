"""Device errors reach the caller: a bounded device wait that runs out (the
self-test kernel waits on an mbarrier and a grid-barrier counter that nothing
signals) is returned as MAP_ERR_TIMEOUT by the handle's next checking call,
the flag is cleared, and the context stays usable.  No fault and no hang: both
waits are poll-limited."""
import numpy as np
import pytest

import oracle
from paper_2512_13319_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_13319_gb300 import build
    build.build()


def setup(T=1000, prec="fp64"):
    from paper_2512_13319_gb300 import MapSmoother
    model = synth.wiener_velocity(2, q=1.0, r=0.1)
    _, y = synth.simulate(model, T, 0.01, seed=3)
    sm = MapSmoother(model, T, 0.01, precision=prec)
    yt = torch.tensor(y, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    return model, y, sm, yt


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_timeout_is_returned_by_the_next_solve_then_cleared():
    from paper_2512_13319_gb300._binding import MAP_ERR_TIMEOUT, MapError
    model, y, sm, yt = setup()
    sm.solve(yt)
    sm.wait_selftest(1000)
    torch.cuda.synchronize()
    with pytest.raises(MapError) as ei:
        sm.solve(yt)
    assert ei.value.status == MAP_ERR_TIMEOUT
    # cleared: the next solve runs and is right
    x = sm.solve(yt).cpu().numpy()
    assert rel(x, oracle.smooth_lti(model, y, 0.01)) < 1e-9
    # both waits of the self-test were counted
    assert sm.stats()[2] == 2
    sm.close()


def test_synchronising_calls_check_after_their_synchronisation():
    from paper_2512_13319_gb300._binding import MAP_ERR_TIMEOUT, MapError
    model, y, sm, yt = setup(prec="fp32")
    sm.wait_selftest(500)
    with pytest.raises(MapError) as ei:
        sm.stats()                       # synchronises, then reports
    assert ei.value.status == MAP_ERR_TIMEOUT
    assert sm.stats() == (0, 0, 2)
    sm.wait_selftest(500)
    yh = torch.tensor(y, dtype=torch.float32).pin_memory()
    with pytest.raises(MapError) as ei:
        sm.solve_host(yh)
    assert ei.value.status == MAP_ERR_TIMEOUT
    x = sm.solve_host(yh).numpy()
    assert rel(x, oracle.smooth_lti(model, y, 0.01)) < 1e-4
    sm.close()


def test_selftest_argument_checks():
    from paper_2512_13319_gb300._binding import MAP_ERR_INVALID_ARG, MapError
    _, _, sm, yt = setup()
    for polls in (0, -1, (1 << 20) + 1):
        with pytest.raises(MapError) as ei:
            sm.wait_selftest(polls)
        assert ei.value.status == MAP_ERR_INVALID_ARG
    sm.solve(yt)
    assert sm.stats() == (0, 0, 0)
    sm.close()
