"""st_smooth_static: smoothing steps for callers that cannot allocate device
memory (their memory pool owns the GPU, or an allocation would stall a
real-time loop).  It must give the same result as st_smooth on an ordinary
handle while working from a host-only handle and the library's static device
work space.  Kept in its own file so that it runs after every other test."""
import numpy as np
import pytest

from paper_1802_09277_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    import os
    from paper_1802_09277_gb300 import build, st as stmod
    if not os.path.exists(stmod.LIB_PATH):
        build.build()
    stmod.load()
    assert torch.cuda.is_available()
    return stmod


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("d,spans,p,N,ne", [(2, (20, 17), 2, 8, 2), (3, (7, 6, 5), 3, 3, 2),
                                            (1, (40,), 1, 5, 3)])
def test_smooth_static_matches_smooth(st, d, spans, p, N, ne):
    ref = st.Solver(d, p, spans, N, ne_per_slab=ne)                  # allocating handle
    host = st.Solver(d, p, spans, N, ne_per_slab=ne, host_only=True)  # no device memory
    u0 = inputs.uniform_vector(50, ref.ndofs)
    f = _dev(inputs.uniform_vector(51, ref.ndofs))
    u_ref, u_static = _dev(u0), _dev(u0)
    for _ in range(2):  # two calls in a row
        ref.smooth(u_ref, f, 1)
        host.smooth_static(u_static, f, 1)
        torch.cuda.synchronize()
        a, b = u_static.cpu().numpy(), u_ref.cpu().numpy()
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()
    ref.close()
    host.close()


def test_smooth_static_rejects_oversize(st):
    host = st.Solver(2, 2, (64, 64), 64, host_only=True)  # 1 048 576 dofs > static limit
    u = torch.zeros(host.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(st.StError) as e:
        host.smooth_static(u, torch.zeros_like(u), 1)
    assert e.value.code == -1


@pytest.mark.parametrize("opts", [dict(variant="eig"), dict(variant="cschur"),
                                  dict(spatial_solver="minres")])
def test_smooth_static_rejects_other_variants(st, opts):
    # the diagonalisation, complex-Schur and MinRes smoothers need device
    # tables the static array does not hold: refused before any copy or launch
    host = st.Solver(2, 2, (12, 10), 4, host_only=True, **opts)
    u = torch.zeros(host.ndofs, dtype=torch.float64, device="cuda")
    f = torch.ones_like(u)
    with pytest.raises(st.StError) as e:
        host.smooth_static(u, f, 1)
    assert e.value.code == -9
    torch.cuda.synchronize()
    assert float(u.abs().max()) == 0.0  # nothing ran
    host.close()
