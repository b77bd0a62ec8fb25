"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64 rounding of sums of O(10)-O(100) terms, written per test):
operator/load/residual 1e-13 relative to the largest output entry; one
smoothing step and one V-cycle 1e-11 (the d spatial transforms and the time
transforms add O(n) rounded terms each); FP64 solve 1e-10 (solved to 1e-12);
mixed-precision solve 1e-8 (solved to 1e-10)."""
import numpy as np
import pytest

from oracle import assemble as A
from oracle import solve as S
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


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


_HIER = {}


def hierarchy(pr):
    """Oracle multigrid hierarchy, cached per problem (the Galerkin products
    dominate the CPU time of the V-cycle tests)."""
    key = (pr.d, pr.spans, pr.p, pr.ne, pr.N, pr.theta)
    if key not in _HIER:
        _HIER[key] = S.Hierarchy(pr)
    return _HIER[key]


def exact(pr, f):
    """The oracle's exact solution by block forward substitution (pinned
    against the sparse-LU solve of the whole system)."""
    return S.forward_subst(pr, f)


# (d, spans, p, N, ne): several tiles per axis and ragged tails (tile sizes
# are 128 (1D), 32x16 (2D), 16x8x4 (3D))
CASES = [
    (1, (16,), 2, 8, 4),       # the 1D manufactured-solution configuration
    (1, (300,), 3, 3, 2),      # 1D, 3 x-tiles ragged, odd slab count
    (2, (8, 6), 3, 5, 2),
    (2, (37, 29), 2, 6, 2),    # 2 x-tiles, 2 y-tiles, ragged
    (2, (20, 20), 1, 4, 5),    # p = 1, nt = 6
    (3, (5, 4, 6), 1, 4, 3),
    (3, (19, 11, 9), 2, 2, 2),  # 3D ragged in every axis
    (3, (6, 6, 6), 3, 2, 2),
]


@pytest.mark.parametrize("d,spans,p,N,ne", CASES)
def test_apply_residual_load_parity(st, d, spans, p, N, ne):
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    L = A.assemble_L(pr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne)
    x = inputs.uniform_vector(1, pr.ndofs)
    f = inputs.uniform_vector(2, pr.ndofs)
    y = torch.empty(pr.ndofs, dtype=torch.float64, device="cuda")
    s.apply(dev(x), y)
    assert relerr(host(y), L @ x) <= 1e-13
    s.residual(dev(x), dev(f), y)
    assert relerr(host(y), f - L @ x) <= 1e-13
    s.load_coeffs(dev(x), y)
    assert relerr(host(y), A.load_from_coeffs(pr, x)) <= 1e-13
    s.close()


@pytest.mark.parametrize("d,spans,p,N,ne", CASES)
def test_smooth_step_parity(st, d, spans, p, N, ne):
    """One damped block-Jacobi step (Sec. 3.1) with A^{-1} by Eq. 3.1 + fast
    diagonalisation equals the oracle's step with sparse-LU slab solves."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    L = A.assemble_L(pr)
    lev = S.Level(L, N, pr.Nt * pr.Nx)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne)
    u0 = inputs.uniform_vector(3, pr.ndofs)
    f = inputs.uniform_vector(4, pr.ndofs)
    ref = S.jacobi_step(lev, u0, f, 0.5)
    u = dev(u0)
    s.smooth(u, dev(f), 1)
    assert relerr(host(u), ref) <= 1e-11
    ref2 = S.jacobi_step(lev, ref, f, 0.5)
    s.smooth(u, dev(f), 1)
    assert relerr(host(u), ref2) <= 1e-11
    s.close()


@pytest.mark.parametrize("basis", ["nodal", "spectral"])
@pytest.mark.parametrize("d,spans,p,N,ne", [c for c in CASES if c[3] > 1])
def test_vcycle_parity(st, basis, d, spans, p, N, ne):
    """One V-cycle (time coarsening, Galerkin coarse operators in the oracle,
    frozen-delta rediscretisation on the GPU) from a nonzero start, in the
    B-spline basis and in the spatial eigenbasis."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    H = hierarchy(pr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, basis=basis)
    u0 = inputs.uniform_vector(5, pr.ndofs)
    f = inputs.uniform_vector(6, pr.ndofs)
    ref = S.vcycle(H, f, u=u0.copy())
    u = dev(u0)
    s.vcycle(u, dev(f))
    assert relerr(host(u), ref) <= 1e-11
    # a second cycle must not depend on state left by the first
    ref2 = S.vcycle(H, f, u=ref.copy())
    s.vcycle(u, dev(f))
    assert relerr(host(u), ref2) <= 1e-11
    s.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 2), (0, 1), (1, 0), (2, 1), (3, 3), (4, 2), (6, 5)])
@pytest.mark.parametrize("d,spans,p,N,ne", [(1, (16,), 2, 64, 2), (2, (6, 5), 2, 32, 2),
                                            (2, (7, 6), 3, 12, 2)])
def test_vcycle_levels_and_tail_parity(st, nu1, nu2, d, spans, p, N, ne):
    """Eigenbasis V-cycle with more than 16 slabs (level-wise kernels above
    the one-launch coarse tail), and with nu1, nu2 other than 1 (general
    smoothing-step kernels, no tail), against the oracle's V(nu1, nu2)."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    H = hierarchy(pr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, basis="spectral", nu1=nu1, nu2=nu2)
    u0 = inputs.uniform_vector(15, pr.ndofs)
    f = inputs.uniform_vector(16, pr.ndofs)
    ref = S.vcycle(H, f, nu1=nu1, nu2=nu2, u=u0.copy())
    u = dev(u0)
    s.vcycle(u, dev(f))
    assert relerr(host(u), ref) <= 1e-11
    s.close()


@pytest.mark.parametrize("basis", ["nodal", "spectral"])
@pytest.mark.parametrize("outer", ["fgmres", "mg"])
@pytest.mark.parametrize("d,spans,p,N,ne", CASES[:6])
def test_solve_fp64_parity(st, basis, outer, d, spans, p, N, ne):
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    c = inputs.normal_coeffs(7, pr.ndofs)
    fr = A.load_from_coeffs(pr, c)
    ud = exact(pr, fr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, outer=outer, basis=basis)
    f = torch.empty(pr.ndofs, dtype=torch.float64, device="cuda")
    s.load_coeffs(dev(c), f)
    u = torch.zeros_like(f)
    info = s.solve(f, u, tol=1e-12)
    err = np.linalg.norm(host(u) - ud) / np.linalg.norm(ud)
    assert info["rel_residual"] <= 1e-12
    assert err <= 1e-10, (err, info)
    s.close()


@pytest.mark.parametrize("basis", ["nodal", "spectral"])
@pytest.mark.parametrize("outer", ["fgmres", "mg"])
@pytest.mark.parametrize("d,spans,p,N,ne", CASES[:6])
def test_solve_mixed_parity(st, basis, outer, d, spans, p, N, ne):
    """FP32 V-cycle, FP64 outer residual and update: 1e-8 vs the oracle."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    c = inputs.normal_coeffs(8, pr.ndofs)
    fr = A.load_from_coeffs(pr, c)
    ud = exact(pr, fr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, outer=outer, precision="mixed_fp32",
                  basis=basis)
    f = dev(fr)
    u = torch.zeros_like(f)
    info = s.solve(f, u, tol=1e-10)
    err = np.linalg.norm(host(u) - ud) / np.linalg.norm(ud)
    assert err <= 1e-8, (err, info)
    s.close()


def test_manufactured_1d_solution(st):
    """The 1D configuration: u = sin(pi x) sin(pi t), multigrid iteration to
    1e-10; the GPU solution equals the oracle's direct solution."""
    pr = A.Problem(1, (16,), 2, 4, 8, theta=1.0)
    fr = A.manufactured_load(pr)
    ud = exact(pr, fr)
    s = st.Solver(1, 2, (16,), 8, ne_per_slab=4, outer="mg")
    u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(fr), u, tol=1e-10)
    assert np.linalg.norm(host(u) - ud) <= 1e-9 * np.linalg.norm(ud)
    assert info["iterations"] <= 40
    s.close()


def test_single_slab_exact_in_one_cycle(st):
    pr = A.Problem(2, (9, 7), 2, 2, 1, theta=1.0)
    fr = inputs.normal_coeffs(9, pr.ndofs)
    ud = exact(pr, fr)
    s = st.Solver(2, 2, (9, 7), 1, outer="mg")
    u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(fr), u, tol=1e-12)
    assert info["iterations"] == 1
    assert relerr(host(u), ud) <= 1e-12


@pytest.mark.parametrize("basis", ["nodal", "spectral"])
def test_multi_rhs_equals_single(st, basis):
    """nrhs independent problems solved together give each single solution."""
    d, spans, p, N = 2, (12, 10), 2, 8
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    R = 3
    fs = [inputs.normal_coeffs(20 + r, pr.ndofs) for r in range(R)]
    sb = st.Solver(d, p, spans, N, nrhs=R, basis=basis)
    assert sb.ndofs == R * pr.ndofs
    u = torch.zeros(R * pr.ndofs, dtype=torch.float64, device="cuda")
    sb.solve(dev(np.concatenate(fs)), u, tol=1e-12)
    ub = host(u).reshape(R, -1)
    L = A.assemble_L(pr)
    for r in range(R):
        ud = exact(pr, fs[r])
        assert np.linalg.norm(ub[r] - ud) <= 1e-10 * np.linalg.norm(ud)
    # the operator is block diagonal over rhs
    x = inputs.uniform_vector(30, R * pr.ndofs)
    y = torch.empty_like(u)
    sb.apply(dev(x), y)
    yr = host(y).reshape(R, -1)
    for r in range(R):
        assert relerr(yr[r], L @ x[r * pr.ndofs:(r + 1) * pr.ndofs]) <= 1e-13


def test_zero_rhs(st):
    s = st.Solver(2, 2, (8, 8), 4)
    f = torch.zeros(s.ndofs, dtype=torch.float64, device="cuda")
    u = torch.ones_like(f)
    info = s.solve(f, u, tol=1e-8)
    assert info["iterations"] == 0
    assert float(u.abs().max()) == 0.0


def test_argument_errors(st):
    s = st.Solver(1, 2, (6,), 2)
    x = torch.zeros(s.ndofs, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        s.apply(x, torch.zeros(s.ndofs + 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        s.apply(x, torch.zeros(s.ndofs, dtype=torch.float32, device="cuda"))
    with pytest.raises(st.StError) as e:
        s.apply(x, x)
    assert e.value.code == -1
    with pytest.raises(st.StError) as e:
        s.solve(x, x, tol=1e-8)
    assert e.value.code == -1


def test_hbm_budget_refused(st):
    with pytest.raises(st.StError) as e:
        st.Solver(2, 2, (64, 64), 256, hbm_budget=1 << 20)
    assert e.value.code == -8


def test_full_size_2d_sampled(st):
    """The 2D workload at full size (64x64 spans, p = 2, 256 slabs x 2
    elements, 4.19 M dofs): st_apply checked slab by slab on sampled slabs,
    and the FP64 solve's residual recomputed by the oracle on every slab."""
    d, spans, p, N, ne = 2, (64, 64), 2, 256, 2
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    Ab, Bb = A.slab_blocks(pr)
    m = pr.Nt * pr.Nx
    s = st.Solver(d, p, spans, N, ne_per_slab=ne)
    x = inputs.uniform_vector(40, pr.ndofs)
    y = torch.empty(pr.ndofs, dtype=torch.float64, device="cuda")
    s.apply(dev(x), y)
    yh = host(y)
    X = x.reshape(N, m)
    for n in (0, 1, 97, 255):
        ref = Ab @ X[n] - (Bb @ X[n - 1] if n else 0.0)
        assert relerr(yh[n * m:(n + 1) * m], ref) <= 1e-13
    c = inputs.normal_coeffs(2, pr.ndofs)
    f = torch.empty_like(y)
    s.load_coeffs(dev(c), f)
    u = torch.zeros_like(y)
    info = s.solve(f, u, tol=1e-8)
    U = host(u).reshape(N, m)
    F = A.load_from_coeffs(pr, c).reshape(N, m)
    res2 = 0.0
    for n in range(N):
        r = F[n] - Ab @ U[n] + (Bb @ U[n - 1] if n else 0.0)
        res2 += float(r @ r)
    rel = np.sqrt(res2) / np.linalg.norm(F)
    assert rel <= 1.01e-8, (rel, info)


# the last two: more than 128 modes on the contiguous axis (two 128-row
# accumulator halves) and on the strided axis, with the contraction staged in
# K chunks where the whole of it does not fit in shared memory
TC_CASES = [(1, (16,), 2, 8, 4), (2, (37, 29), 2, 6, 2), (2, (20, 20), 1, 4, 5),
            (3, (19, 11, 9), 2, 2, 2), (2, (64, 64), 2, 4, 2), (2, (130, 20), 2, 4, 2),
            (2, (20, 150), 3, 4, 2)]


@pytest.mark.parametrize("prec,tol", [("mixed_tf32", 1e-2), ("mixed_bf16", 6e-2)])
@pytest.mark.parametrize("d,spans,p,N,ne", TC_CASES)
def test_vcycle_tensor_core_transforms(st, prec, tol, d, spans, p, N, ne):
    """One V-cycle with the spatial transforms on the tensor cores (operands
    rounded to TF32: 10-bit, BF16: 7-bit mantissa; FP32 accumulation) stays
    within a rounding-level distance of the oracle's FP64 V-cycle."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    H = hierarchy(pr)
    f = inputs.uniform_vector(60, pr.ndofs)
    ref = S.vcycle(H, f)
    for basis in ("spectral", "nodal"):
        s = st.Solver(d, p, spans, N, ne_per_slab=ne, precision=prec, basis=basis)
        u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        s.vcycle(u, dev(f))
        assert relerr(host(u), ref) <= tol, (basis, relerr(host(u), ref))
        s.close()


@pytest.mark.parametrize("prec", ["mixed_tf32", "mixed_bf16"])
@pytest.mark.parametrize("d,spans,p,N,ne", TC_CASES)
def test_solve_tensor_core_parity(st, prec, d, spans, p, N, ne):
    """FGMRES with the tensor-core V-cycle reaches the oracle's solution to
    1e-8: the FP64 outer residual recovers the accuracy of the TF32 / BF16
    transforms."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    c = inputs.normal_coeffs(61, pr.ndofs)
    fr = A.load_from_coeffs(pr, c)
    ud = exact(pr, fr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, precision=prec, basis="spectral")
    u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(fr), u, tol=1e-10)
    err = np.linalg.norm(host(u) - ud) / np.linalg.norm(ud)
    assert err <= 1e-8, (err, info)
    s.close()


@pytest.mark.parametrize("prec", ["mixed_fp32", "mixed_tf32", "mixed_bf16"])
@pytest.mark.parametrize("basis", ["spectral", "nodal"])
@pytest.mark.parametrize("d,spans,p,N,ne", [CASES[0], CASES[3], CASES[5], (2, (64, 64), 2, 8, 2)])
def test_solve_refinement_parity(st, prec, basis, d, spans, p, N, ne):
    """Mixed-precision iterative refinement (FP64 residual and update around
    FP32 FGMRES with FP32 operator and V-cycle) reaches the oracle to 1e-8."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    c = inputs.normal_coeffs(62, pr.ndofs)
    fr = A.load_from_coeffs(pr, c)
    ud = exact(pr, fr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, precision=prec, basis=basis, outer="ir")
    u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(fr), u, tol=1e-10)
    err = np.linalg.norm(host(u) - ud) / np.linalg.norm(ud)
    assert err <= 1e-8, (err, info)
    assert info["refinements"] >= 1
    s.close()


@pytest.mark.parametrize("d,spans,p,N,ne", [CASES[3], (2, (64, 64), 2, 8, 2), (3, (10, 9, 8), 2, 4, 2),
                                            (2, (130, 20), 2, 4, 2), (2, (20, 150), 3, 4, 2)])
def test_split_tf32_transforms_keep_fp32_refinement(st, d, spans, p, N, ne):
    """In the eigenbasis refinement only the two spatial transforms around
    each inner solve leave the eigenbasis; on the tensor cores they run as
    split TF32 (hi*hi + hi*lo + lo*hi).  Their error must stay at the FP32
    level: the refinement then takes no more steps than with FP32 CUDA-core
    transforms, and its result matches the oracle."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    c = inputs.normal_coeffs(63, pr.ndofs)
    fr = A.load_from_coeffs(pr, c)
    ud = exact(pr, fr)
    refs = {}
    for prec in ("mixed_fp32", "mixed_tf32", "mixed_bf16"):
        s = st.Solver(d, p, spans, N, ne_per_slab=ne, precision=prec, basis="spectral", outer="ir")
        u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        info = s.solve(dev(fr), u, tol=1e-11)
        s.close()
        err = np.linalg.norm(host(u) - ud) / np.linalg.norm(ud)
        assert err <= 1e-9, (prec, err, info)
        refs[prec] = info["refinements"]
    assert refs["mixed_tf32"] <= refs["mixed_fp32"], refs
    assert refs["mixed_bf16"] <= refs["mixed_fp32"], refs


def test_refinement_multi_rhs_equals_single(st):
    d, spans, p, N = 2, (12, 10), 2, 8
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    R = 3
    fs = [inputs.normal_coeffs(70 + r, pr.ndofs) for r in range(R)]
    sb = st.Solver(d, p, spans, N, nrhs=R, precision="mixed_tf32", basis="spectral", outer="ir")
    u = torch.zeros(R * pr.ndofs, dtype=torch.float64, device="cuda")
    sb.solve(dev(np.concatenate(fs)), u, tol=1e-10)
    ub = host(u).reshape(R, -1)
    L = A.assemble_L(pr)
    for r in range(R):
        s1 = st.Solver(d, p, spans, N, precision="mixed_tf32", basis="spectral", outer="ir")
        u1 = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        s1.solve(dev(fs[r]), u1, tol=1e-10)
        # each rhs is refined independently: the batched result is the single one
        assert np.array_equal(host(u1), ub[r])
        ud = exact(pr, fs[r])
        assert np.linalg.norm(ub[r] - ud) <= 1e-8 * np.linalg.norm(ud)


@pytest.mark.parametrize("basis", ["nodal", "spectral"])
@pytest.mark.parametrize("d,spans,p,N,ne", [CASES[0], CASES[2], CASES[3], CASES[5]])
@pytest.mark.parametrize("variant", ["eig", "cschur"])
def test_eig_variant_vcycle_and_solve(st, variant, basis, d, spans, p, N, ne):
    """Diagonalisation variant (Sec. 3.3, complex shifts) and complex Schur
    variant (Sec. 3.4, Algorithm 1: complex triangular solve): one smoothing
    step, one V-cycle and an FP64 solve equal the oracle's."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    H = hierarchy(pr)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, variant=variant, basis=basis)
    u0 = inputs.uniform_vector(80, pr.ndofs)
    f = inputs.uniform_vector(81, pr.ndofs)
    u = dev(u0)
    s.smooth(u, dev(f), 1)
    lev = S.Level(H.levels[0].L, N, pr.Nt * pr.Nx)
    assert relerr(host(u), S.jacobi_step(lev, u0, f, 0.5)) <= 1e-10
    if N > 1:
        u = dev(u0)
        s.vcycle(u, dev(f))
        assert relerr(host(u), S.vcycle(H, f, u=u0.copy())) <= 1e-10
    ud = exact(pr, f)
    x = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
    s.solve(dev(f), x, tol=1e-12)
    assert np.linalg.norm(host(x) - ud) <= 1e-10 * np.linalg.norm(ud)
    s.close()


@pytest.mark.parametrize("d,spans,p,N,ne", [(1, (16,), 2, 8, 4), (2, (12, 9), 3, 4, 2),
                                            (3, (5, 6, 4), 2, 3, 2)])
def test_gaussian_bump_load_parity(st, d, spans, p, N, ne):
    """Space-time Gaussian-bump source: library quadrature vs the oracle's
    (both Gauss-Legendre, 2p + 4 points per element)."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    cen, wid, amp = inputs.gaussian_bumps(9, count=6, dim=d + 1)
    ref = A.bumps_load(pr, cen, wid, amp)
    s = st.Solver(d, p, spans, N, ne_per_slab=ne)
    f = torch.empty(pr.ndofs, dtype=torch.float64, device="cuda")
    s.load_gaussians(cen, wid, amp, f)
    assert relerr(host(f), ref) <= 1e-13
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
@pytest.mark.parametrize("d,spans,p,N,ne", [CASES[0], CASES[3], CASES[4], CASES[6], (2, (64, 64), 2, 64, 2)])
def test_fused_vcycle_matches_levelwise(st, prec, d, spans, p, N, ne):
    """The one-kernel shared-memory V-cycle gives the level-by-level
    eigenbasis V-cycle's result, and both match the oracle's V-cycle."""
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    f = inputs.uniform_vector(90, pr.ndofs)
    out = []
    for fused in (1, 0):
        s = st.Solver(d, p, spans, N, ne_per_slab=ne, precision=prec, basis="spectral",
                      fused_vcycle=fused)
        u = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        s.vcycle(u, dev(f))
        out.append(host(u))
        s.close()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert relerr(out[0], out[1]) <= tol
    if pr.ndofs > 300000:  # the level-wise cycle is pinned to the oracle at the smaller sizes
        return
    ref = S.vcycle(hierarchy(pr), f)
    assert relerr(out[0], ref) <= (1e-11 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec,outer,basis", [("fp64", "fgmres", "nodal"), ("fp64", "mg", "nodal"),
                                              ("mixed_tf32", "ir", "spectral")])
def test_solve_history(st, prec, outer, basis):
    """st_solve_history: the FP64 relative residual at every restart /
    multigrid iteration / refinement; it starts at 1 (zero initial guess),
    ends at the solve's reported residual and decreases overall."""
    d, spans, p, N = 2, (16, 12), 2, 8
    pr = A.Problem(d, spans, p, 2, N, theta=1.0)
    s = st.Solver(d, p, spans, N, precision=prec, outer=outer, basis=basis, gmres_restart=5)
    f = dev(inputs.uniform_vector(77, pr.ndofs))
    u = torch.zeros_like(f)
    info = s.solve(f, u, tol=1e-10)
    hist = s.history()
    assert len(hist) >= 2
    assert abs(hist[0][1] - 1.0) <= 1e-12 and hist[0][0] == 0
    assert hist[-1][1] == info["rel_residual"] and hist[-1][0] == info["iterations"]
    assert hist[-1][1] <= 1e-10 < hist[0][1]
    assert all(b[0] >= a[0] for a, b in zip(hist, hist[1:]))
    s.close()


@pytest.mark.parametrize("spans,p", [((18, 5, 67), 2), ((9, 4, 70), 3)])
def test_refinement_residual_3d_z_chunks(st, spans, p):
    """The FP64-accurate refinement residual of the 3D mixed solve with more
    than 64 z planes: at p = 3 the z-marching kernel in chunks of 32 planes
    (ragged last chunk), at p = 2 the tiled kernel (ragged tiles in every
    axis); the refined solution matches the oracle's direct one."""
    d, N, ne = 3, 2, 2
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    c = inputs.normal_coeffs(91, pr.ndofs)
    ud = exact(pr, A.load_from_coeffs(pr, c))
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, precision="mixed_tf32", basis="spectral",
                  outer="ir")
    f = torch.empty(pr.ndofs, dtype=torch.float64, device="cuda")
    s.load_coeffs(dev(c), f)
    u = torch.zeros_like(f)
    info = s.solve(f, u, tol=1e-10)
    err = np.linalg.norm(host(u) - ud) / np.linalg.norm(ud)
    assert info["rel_residual"] <= 1e-10 and err <= 1e-8, (err, info)
    s.close()


def test_refinement_many_modes_register_tail(st):
    """With many (mode, right-hand side) pairs and V(4,4) the eigenbasis
    V-cycle sweeps down to 4 slabs and ends in the register-resident tail
    (a 16-slab tail would spill its vectors out of L1): 16 right-hand sides
    of a 64 x 64, p = 2 problem on 16 slabs reach the oracle's solution to
    1e-8, and match the solves of one right-hand side each (which end in
    the 16-slab tail) to the same tolerance."""
    d, spans, p, N, ne, R = 2, (64, 64), 2, 16, 2, 16
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    cs = [inputs.normal_coeffs(90 + r, pr.ndofs) for r in range(R)]
    F = [A.load_from_coeffs(pr, c) for c in cs]
    s = st.Solver(d, p, spans, N, ne_per_slab=ne, nrhs=R, precision="mixed_tf32",
                  basis="spectral", outer="ir", nu1=4, nu2=4)
    u = torch.zeros(R * pr.ndofs, dtype=torch.float64, device="cuda")
    info = s.solve(dev(np.concatenate(F)), u, tol=1e-10)
    assert info["rel_residual"] <= 1e-10
    got = host(u).reshape(R, pr.ndofs)
    for r in (0, R - 1):
        ud = exact(pr, F[r])
        assert np.linalg.norm(got[r] - ud) <= 1e-8 * np.linalg.norm(ud), r
    s.close()
    one = st.Solver(d, p, spans, N, ne_per_slab=ne, nrhs=1, precision="mixed_tf32",
                    basis="spectral", outer="ir", nu1=4, nu2=4)
    for r in range(R):
        u1 = torch.zeros(pr.ndofs, dtype=torch.float64, device="cuda")
        one.solve(dev(F[r]), u1, tol=1e-10)
        v = host(u1)
        assert np.linalg.norm(got[r] - v) <= 1e-8 * np.linalg.norm(v), r
    one.close()
