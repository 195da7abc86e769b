"""The allocation-free G* entry point, for callers that cannot allocate
device memory (an application whose own pool owns all device memory, a
plug-in inside a framework that does): it must give the same result as the
handle-based rve_op_apply_gamma, call after call, and reject grids larger
than its static scratch.  Collected last (file name), so a run that stops at
the first failure has run every other test first."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_04770_gb300 as p
    p.lib()
    return p


@pytest.mark.parametrize("n,ctrl", [((32, 24, 16), [1, 0, 0, 0, 0, 0]),
                                    ((64, 48), [1, 0, 1, 1, 1, 0]),
                                    ((64, 64, 64), [1, 1, 1, 1, 1, 1])])
def test_noalloc_gamma_matches_handle_entry_point(pkg, n, ctrl):
    dim = len(n)
    nc = 6 if dim == 3 else 3
    V = int(np.prod(n))
    L = [float(x) * 0.5 for x in n]
    rng = np.random.default_rng(11)
    h = pkg.rve_create(dim, n, L, pkg.RVE_FP64, 1)
    try:
        pkg.rve_set_phases(h, np.zeros(tuple(reversed(n)), dtype=np.uint8),
                           [dict(E=1000.0, nu=0.3), dict(E=2000.0, nu=0.2)], np.array([[1.0, 0.1]]))
        pkg.rve_set_load_path(h, ctrl, np.zeros((1, 6)))
        for call in range(2):                      # two calls in a row share the scratch
            tau = torch.as_tensor(rng.standard_normal((nc, V)) + 0.5 * call, device="cuda")
            ref = torch.empty(nc, V, device="cuda", dtype=torch.float64)
            pkg.rve_op_apply_gamma(h, tau, ref)
            out = torch.full((nc, V), float("nan"), device="cuda", dtype=torch.float64)
            pkg.rve_op_apply_gamma_noalloc(dim, n, L, ctrl, tau, out)
            scale = float(tau.abs().max())
            assert float((out - ref).abs().max()) <= 1e-12 * scale
    finally:
        pkg.rve_free(h)


def test_noalloc_rejects_grids_beyond_the_scratch(pkg):
    n = (96, 96, 96)
    V = int(np.prod(n))
    tau = torch.zeros(6, 8, device="cuda", dtype=torch.float64)   # never touched
    with pytest.raises(pkg.RVEError) as e:
        pkg.rve_op_apply_gamma_noalloc(3, n, [96.0] * 3, [1] * 6, tau, tau)
    assert e.value.status == pkg.RVE_ERR_ARG
    assert V > 0
