"""The timeout path of the 3D projection pass's tile copies, exercised
without a fault: the test hook adds bytes that no copy delivers to the count
the tile barrier expects, so every CTA's wait runs out (after 1 ms) although
its copy lands.  The call must report RVE_ERR_TIMEOUT, and the device must
stay usable: a fresh handle then computes G* as before."""
import numpy as np
import pytest

import rve_inputs as I
from oracle import rve_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_04770_gb300 as p
    p.lib()
    return p


def _handle(pkg, n):
    h = pkg.rve_create(3, n, [float(x) for x in n], pkg.RVE_FP64, 1)
    pkg.rve_set_phases(h, np.zeros(tuple(reversed(n)), dtype=np.uint8), [I.MATRIX, I.PARTICLE],
                       np.array([[1.0, 0.02]]))
    return h


def test_tile_wait_timeout_is_reported_and_the_device_stays_usable(pkg):
    n = (16, 12, 64)              # 64-point last axis, six components: TMA tiles
    g = O.Grid(n)
    V = g.V
    rng = np.random.default_rng(4)
    tau = rng.standard_normal(g.shape + (6,))
    tau_d = torch.as_tensor(np.ascontiguousarray(tau.reshape(V, 6).T), device="cuda")
    out = torch.empty(6, V, device="cuda", dtype=torch.float64)
    h = _handle(pkg, n)
    try:
        pkg.rve_test_tile_wait(h, 1e-3, 64)
        with pytest.raises(pkg.RVEError) as e:
            pkg.rve_op_apply_gamma(h, tau_d, out)
        assert e.value.status == pkg.RVE_ERR_TIMEOUT
    finally:
        pkg.rve_free(h)
    torch.cuda.synchronize()
    h = _handle(pkg, n)
    try:
        pkg.rve_op_apply_gamma(h, tau_d, out)
        ref = O.G_apply(tau, g, np.zeros(6))
        got = out.cpu().numpy().T.reshape(g.shape + (6,))
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    finally:
        pkg.rve_free(h)


def test_tile_wait_hook_rejects_bad_arguments(pkg):
    h = _handle(pkg, (8, 8, 64))
    try:
        for args in ((0.0, 0), (100.0, 0), (1.0, -1), (1.0, 1 << 20)):
            with pytest.raises(pkg.RVEError):
                pkg.rve_test_tile_wait(h, *args)
    finally:
        pkg.rve_free(h)
