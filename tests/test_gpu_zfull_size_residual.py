"""The double-float refinement residual (st_residual_df) at the full size of
the 3D workload, in the launch configuration the benchmark times, against the
CPU oracle on sampled slabs.  (The file name puts it after the other GPU
parity files: it holds about 22 GB of vectors while it runs.)

Tolerance as in tests/test_gpu_residual_df.py: entry i may be off by 1e-13 of
the size of the terms it sums, |f_n| + (|K_t| (x) |M_x| + |M_t| (x) |K_x|)|u_n|
+ (|N_t| (x) |M_x|)|u_{n-1}| (about 28 units of 2^-48)."""
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


def _sampled_slab_errors(pr, R, x, f, r, picks):
    """Largest |r - r_oracle| / (size of the residual's terms) over the
    sampled (rhs, slab) pairs, with the oracle's block row of Eq. 2.4 applied
    factor by factor; x, f, r: torch tensors of all right-hand sides."""
    N = pr.N
    m = pr.Nt * pr.Nx

    def sl(v, q, n):
        return v[(q * N + n) * m:(q * N + n + 1) * m].cpu().numpy()

    worst = 0.0
    for q in sorted({0, R - 1}):
        for n in picks:
            up = sl(x, q, n - 1) if n else None
            ref = A.slab_residual_kron(pr, sl(f, q, n), sl(x, q, n), up)
            scale = A.slab_residual_kron(pr, sl(f, q, n), sl(x, q, n), up, magnitude=True)
            worst = max(worst, float((np.abs(sl(r, q, n) - ref) / scale).max()))
    return worst


def test_residual_df_full_size_sampled(st):
    """48^3 spans, p = 2, 128 slabs x 2 elements, 16 right-hand sides solved
    together (906 M dofs; the library picks 8 slabs per CTA, as in the
    benchmark's solve): slabs at the starts and ends of the CTAs' 8-slab
    chunks (a recomputed and a carried coupling plane) and at the start of
    each problem (no coupling), of the first and last right-hand side."""
    d, spans, p, N, ne, R = 3, (48, 48, 48), 2, 128, 2, 16
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, nrhs=R, precision="mixed_tf32",
                  basis="spectral", outer="ir")
    assert s.ndofs == R * pr.ndofs
    x, f = inputs.uniform_vectors_on_device(77, s.ndofs, 2, "cuda")
    r = torch.empty_like(x)
    s.residual_df(x, f, r)
    torch.cuda.synchronize()
    s.close()
    worst = _sampled_slab_errors(pr, R, x, f, r, (0, 1, 7, 8, 9, 63, 64, 120, 127))
    del x, f, r
    torch.cuda.empty_cache()
    print("residual_df 48^3 x 128 slabs x 16 rhs: max |r - r_oracle| / terms = %.2e" % worst)
    assert worst <= 1e-13
