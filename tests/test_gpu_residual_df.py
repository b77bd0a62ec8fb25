"""GPU parity of the double-float residual (st_residual_df: the FP64-accurate
residual r = f - L u of the mixed-precision iterative refinement, Eq. 2.4
through the Kronecker factors of Eq. 2.5) against the CPU oracle's assembled
L_h, element by element.

Tolerance: every input and coefficient is held to about 48 significant bits
(2^-48 = 3.6e-15) and every sum-factorised pass rounds its results to that
precision, so entry i is off by at most a small multiple of
2^-48 (|L| |u| + |f|)_i, |L| the entry-wise absolute value of the assembled
operator; the test allows 1e-13 (about 28 units of 2^-48) of that, and 1e-12
relative to the largest output entry.

The tiled kernel lets one CTA handle several consecutive slabs and take the
coupling plane of its later slabs from the slab before; the result must not
depend on how many (ragged last chunks and problem boundaries inside a
chunk included)."""
import numpy as np
import pytest

from oracle import assemble as A
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


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# (d, spans, p, N, ne, nrhs): several tiles per axis with ragged tails (tiled
# kernel tiles: 128 (1D), 32 x 16 (2D), 8 x 8 x 16 (3D)); slab counts that
# leave ragged chunks of 2, 4 and 8 slabs; several right-hand sides, so that
# chunks cross the boundary between two problems (no coupling there); the 3D
# p = 3 case runs the z-marching kernel
CASES = [
    (1, (16,), 2, 8, 4, 1),
    (1, (300,), 3, 3, 2, 2),
    (2, (8, 6), 3, 5, 2, 3),
    (2, (37, 29), 2, 6, 2, 1),
    (2, (20, 20), 1, 4, 5, 1),
    (2, (33, 17), 2, 7, 2, 2),
    (3, (5, 4, 6), 1, 4, 3, 1),
    (3, (19, 11, 9), 2, 3, 2, 3),
    (3, (6, 6, 6), 3, 2, 2, 2),
]


@pytest.mark.parametrize("d,spans,p,N,ne,R", CASES)
def test_residual_df_parity(st, d, spans, p, N, ne, R):
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    L = A.assemble_L(pr)
    absL = abs(L)
    n = pr.ndofs
    x = np.concatenate([inputs.uniform_vector(10 + q, n) for q in range(R)])
    f = np.concatenate([inputs.uniform_vector(20 + q, n) for q in range(R)])
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, nrhs=R)
    xd, fd = dev(x), dev(f)
    r = torch.empty(R * n, dtype=torch.float64, device="cuda")
    got = {}
    for spc in (0, 1, 2, 4, 8):
        r.fill_(np.nan)
        s.residual_df(xd, fd, r, slabs_per_cta=spc)
        got[spc] = host(r).copy()
    s.close()
    worst = 0.0
    for q in range(R):
        xq, fq = x[q * n:(q + 1) * n], f[q * n:(q + 1) * n]
        ref = fq - L @ xq
        scale = absL @ np.abs(xq) + np.abs(fq)
        err = np.abs(got[1][q * n:(q + 1) * n] - ref)
        worst = max(worst, float((err / scale).max()))
        assert (err <= 1e-13 * scale).all(), (q, float((err / scale).max()))
        assert err.max() <= 1e-12 * np.abs(ref).max()
    print("residual_df d=%d p=%d N=%d R=%d: max |r - r_oracle| / (|L||u| + |f|) = %.2e"
          % (d, p, N, R, worst))
    for spc in (0, 2, 4, 8):  # one slab per CTA or several: the same bits
        assert np.array_equal(got[spc], got[1]), spc


def test_residual_df_on_mixed_handle_and_errors(st):
    """A mixed-precision eigenbasis handle (the refinement's own) gives the
    FP64 handle's bits; invalid arguments are refused before any launch."""
    d, spans, p, N, ne = 2, (37, 29), 2, 6, 2
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    x = dev(inputs.uniform_vector(31, pr.ndofs))
    f = dev(inputs.uniform_vector(32, pr.ndofs))
    outs = []
    for kw in (dict(), dict(precision="mixed_tf32", basis="spectral", outer="ir")):
        s = st.Solver(d, p, spans, N, ne_per_slab=ne, **kw)
        r = torch.empty_like(x)
        s.residual_df(x, f, r)
        outs.append(host(r))
        if kw:
            for bad in (3, -1, 16):
                with pytest.raises(st.StError) as e:
                    s.residual_df(x, f, r, slabs_per_cta=bad)
                assert e.value.code == st.ST_ERR_INVALID_ARG
            with pytest.raises(st.StError) as e:
                s.residual_df(x, f, x)  # r aliases u
            assert e.value.code == st.ST_ERR_INVALID_ARG
        s.close()
    assert np.array_equal(outs[0], outs[1])

