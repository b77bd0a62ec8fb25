"""Failure handling on the GPU without a GPU fault: a bounded device wait
that runs out is reported as ST_ERR_TIMEOUT and leaves the handle usable;
a right-hand side with NaN entries is rejected as an argument error."""
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


def test_tensor_core_wait_runs_out_and_handle_recovers(st):
    # B-spline-basis V-cycle with its spatial transforms on the tensor cores
    d, spans, p, N = 2, (37, 29), 2, 8
    s = st.Solver(d, p, spans, N, precision="mixed_tf32", basis="nodal", outer="fgmres")
    f = _dev(inputs.uniform_vector(31, s.ndofs))
    u = torch.zeros_like(f)
    s.set_wait_limit(0.0)  # every wait for the MMAs is a single test of the signal
    with pytest.raises(st.StError) as e:
        s.vcycle(u, f)
    assert e.value.code == -6  # ST_ERR_TIMEOUT
    # the context and the handle still work: the same cycle with the default
    # bound gives a fresh handle's result
    s.set_wait_limit(1.0)
    u.zero_()
    s.vcycle(u, f)
    ref = st.Solver(d, p, spans, N, precision="mixed_tf32", basis="nodal", outer="fgmres")
    u2 = torch.zeros_like(f)
    ref.vcycle(u2, f)
    torch.cuda.synchronize()
    assert torch.equal(u, u2)
    s.close()
    ref.close()
    with pytest.raises(st.StError):
        st.Solver(d, p, spans, N).set_wait_limit(-1.0)


@pytest.mark.parametrize("prec,outer", [("fp64", "fgmres"), ("mixed_tf32", "ir"), ("fp64", "mg")])
def test_nan_rhs_is_rejected(st, prec, outer):
    s = st.Solver(2, 2, (10, 10), 4, precision=prec, outer=outer, basis="spectral"
                  if outer == "ir" else "nodal")
    f = _dev(inputs.uniform_vector(32, s.ndofs))
    f[123] = float("nan")
    u = torch.zeros_like(f)
    with pytest.raises(st.StError) as e:
        s.solve(f, u, tol=1e-8)
    assert e.value.code == -1
    s.close()
