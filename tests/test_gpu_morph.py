"""GPU parity of the morphing transform entry points (fftenkf_morph_*, Sec. 2.2) against the FP64
oracle in oracle/morph.py, through the C ABI: the forward transform (fixed-point inverse mapping),
the reference mean, the inverse transform, the data's transform, integer shifts (exact), a
morphing FFT EnKF analysis chained through the library, and sampled nodes at 4096^2, K = 20.
FP32 throughout; tolerance 1e-5 relative L2 (FP32 rounding of unit-scale fields and offsets of a
few cells), max abs 1e-4."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import enkf, morph  # noqa: E402
from synth import fields  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5
ATOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1001_1588_gb300 import abi
    abi.lib()


def _abi():
    from paper_1001_1588_gb300 import abi
    return abi


def _rel(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _inputs(M, K, ny, nx, amp, seed):
    u = fields.smooth_members(seed, M, K, ny, nx, ell=8.0)
    u_ref = fields.smooth_members(seed + 1, M, 1, ny, nx, ell=8.0)[:, 0]
    T = fields.smooth_mappings(seed + 2, K, ny, nx, amp=amp, ell=10.0)
    return u, u_ref, T


def _gpu_forward(u, u_ref, T, n_iter, tol=0.0):
    M, K, ny, nx = u.shape
    ext = torch.zeros((M + 2, K, ny, nx), dtype=torch.float32, device="cuda")
    ext[:2] = _dev(T)
    _abi().fftenkf_morph_forward(_dev(u), _dev(u_ref), ext, M, K, ny, nx, n_iter, tol)
    torch.cuda.synchronize()
    return ext.cpu().numpy()


@pytest.mark.parametrize("M,K,ny,nx,n_iter,tol", [(2, 5, 96, 200, 20, 0.0), (1, 3, 37, 61, 8, 0.0),
                                                  (3, 1, 8, 8, 0, 0.0), (2, 4, 128, 160, 20, 1e-5)])
def test_forward_matches_oracle(M, K, ny, nx, n_iter, tol):
    u, u_ref, T = _inputs(M, K, ny, nx, 2.5, 100 + M)
    ext = _gpu_forward(u, u_ref, T, n_iter, tol)
    np.testing.assert_array_equal(ext[:2], T)   # the mappings are left as they were
    ref = morph.morph_forward(u, u_ref, T, n_iter, tol)
    assert _rel(ext[2:], ref) <= TOL
    assert np.abs(ext[2:] - ref).max() <= ATOL


def _lipschitz_inf(f):
    """Max-norm Lipschitz constant of the bilinear interpolant of the periodic field(s) f [..][ny][nx]
    along each axis: the largest node difference (the interpolant's partial derivatives)."""
    f = np.asarray(f, np.float64)
    dx = np.abs(np.roll(f, -1, axis=-1) - f).max()
    dy = np.abs(np.roll(f, -1, axis=-2) - f).max()
    return dx, dy


def test_forward_stopping_rule_near_converged_fixed_point():
    """The kernel stops a point after the first step that moves it by at most tol = 1e-5 cells; the
    oracle's converged inverse mapping (tol = 0, 80 steps: every iterate repeats) is the fixed point
    q* = p - T(q*).  For the iteration map q -> p - T(q) with max-norm Lipschitz constant kappa < 1
    (kappa <= max over components of |dT/dx| + |dT/dy|), a step of size delta <= tol leaves the
    iterate within kappa delta / (1 - kappa) of q*, and the residual r = u(q) - u_ref moves by at most
    |du/dx| + |du/dy| times that.  The GPU residuals must lie within that bound plus the FP32 rounding
    allowance of the other tests (ATOL)."""
    M, K, ny, nx, tol = 2, 4, 128, 160, 1e-5
    u, u_ref, T = _inputs(M, K, ny, nx, 2.5, 211)
    ext = _gpu_forward(u, u_ref, T, 20, tol)
    ref = morph.morph_forward(u, u_ref, T, 80, 0.0)
    kappa = 0.0
    for k in range(K):
        for c in range(2):
            dx, dy = _lipschitz_inf(T[c, k])
            kappa = max(kappa, dx + dy)
    assert kappa < 1.0, kappa
    gu = max(sum(_lipschitz_inf(u[j, k])) for j in range(M) for k in range(K))
    bound = gu * tol * kappa / (1.0 - kappa)
    err = np.abs(ext[2:] - ref).max()
    assert err <= ATOL + bound, (err, bound, kappa)
    assert _rel(ext[2:], ref) <= TOL


def test_forward_integer_shift_exact():
    M, K, ny, nx = 2, 3, 24, 40
    u, u_ref, _ = _inputs(M, K, ny, nx, 1.0, 7)
    T = np.zeros((2, K, ny, nx), np.float32)
    T[0] = 5.0
    T[1] = -3.0
    ext = _gpu_forward(u, u_ref, T, 3)
    want = (np.roll(u, shift=(-3, 5), axis=(2, 3)) - u_ref[:, None]).astype(np.float32)
    np.testing.assert_array_equal(ext[2:], want)


def test_reference_and_inverse_match_oracle():
    M, K, ny, nx = 2, 6, 72, 136
    rng = np.random.default_rng(21)
    u, u_ref, T = _inputs(M, K, ny, nx, 2.0, 300)
    ext = morph.morph_forward(u, u_ref, T, 20)
    ext = np.concatenate([T.astype(np.float64), ext]) + 0.05 * rng.standard_normal((M + 2, K, ny, nx))
    ext = ext.astype(np.float32)
    e = _dev(ext)
    ref_d = torch.empty((M + 2, ny, nx), dtype=torch.float32, device="cuda")
    _abi().fftenkf_morph_reference(e, ref_d, M + 2, K, ny, nx)
    out = torch.empty((M, K, ny, nx), dtype=torch.float32, device="cuda")
    ur = _dev(u_ref)
    _abi().fftenkf_morph_inverse(e, ur, out, M, K, ny, nx)
    out_ref = torch.empty((M, 1, ny, nx), dtype=torch.float32, device="cuda")
    _abi().fftenkf_morph_inverse(ref_d, ur, out_ref, M, 1, ny, nx)
    torch.cuda.synchronize()
    want_ref = morph.morph_reference(ext)
    np.testing.assert_allclose(ref_d.cpu().numpy(), want_ref[:, 0], rtol=0, atol=1e-6)
    want = morph.morph_inverse(ext, u_ref)
    got = out.cpu().numpy()
    assert _rel(got, want) <= TOL and np.abs(got - want).max() <= ATOL
    want_r = morph.morph_inverse(want_ref, u_ref)
    got_r = out_ref.cpu().numpy()
    assert _rel(got_r, want_r) <= TOL and np.abs(got_r - want_r).max() <= ATOL


def test_morphing_enkf_chain_matches_oracle():
    # Sec. 2.2 end to end: transform members and data, FFT EnKF on the extended state with
    # T_x, T_y, r^(1) observed, reference mean, inverse transform; every step in the library.
    from paper_1001_1588_gb300 import torch_api
    M, N, ny, nx = 2, 8, 64, 96
    u, u_ref, T = _inputs(M, N, ny, nx, 2.0, 500)
    d, _, T0 = _inputs(1, 1, ny, nx, 2.0, 600)
    rng = np.random.default_rng(31)
    pert = (0.1 * rng.standard_normal((N, 3, ny, nx))).astype(np.float32)
    rhat = np.full((3, ny, nx // 2 + 1), 0.01, dtype=np.float64)
    observed = np.array([1, 1, 1] + [0] * (M - 1), dtype=np.uint8)
    abi = _abi()
    ext = torch.zeros((M + 2, N, ny, nx), dtype=torch.float32, device="cuda")
    ext[:2] = _dev(T)
    ur = _dev(u_ref)
    abi.fftenkf_morph_forward(_dev(u), ur, ext, M, N, ny, nx, 20, 1e-5)
    data = torch.zeros((3, 1, ny, nx), dtype=torch.float32, device="cuda")
    data[:2] = _dev(T0)
    abi.fftenkf_morph_forward(_dev(d), ur[:1], data, 1, 1, ny, nx, 20, 1e-5)
    plan = torch_api.Plan(ny, nx, M + 2, N, torch.float32, observed)
    plan.analyze(ext, data.reshape(3, ny, nx), _dev(pert), torch.from_numpy(rhat).cuda())
    assert plan.device_status() == 0
    plan.close()
    ext_ref = torch.empty((M + 2, ny, nx), dtype=torch.float32, device="cuda")
    abi.fftenkf_morph_reference(ext, ext_ref, M + 2, N, ny, nx)
    ua = torch.empty((M, N, ny, nx), dtype=torch.float32, device="cuda")
    abi.fftenkf_morph_inverse(ext, ur, ua, M, N, ny, nx)
    ua_ref = torch.empty((M, 1, ny, nx), dtype=torch.float32, device="cuda")
    abi.fftenkf_morph_inverse(ext_ref, ur, ua_ref, M, 1, ny, nx)
    torch.cuda.synchronize()

    e_or = np.concatenate([T.astype(np.float64), morph.morph_forward(u, u_ref, T, 20, 1e-5)])
    d_or = np.concatenate([T0.astype(np.float64), morph.morph_forward(d, u_ref[:1], T0, 20, 1e-5)])[:, 0]
    e_or = enkf.analyze(e_or, d_or, pert, rhat, observed)
    want = morph.morph_inverse(e_or, u_ref)
    want_ref = morph.morph_inverse(morph.morph_reference(e_or), u_ref)
    assert _rel(ua.cpu().numpy(), want) <= 1e-4
    assert _rel(ua_ref.cpu().numpy(), want_ref) <= 1e-4


def test_full_size_sampled_nodes():
    # 4096^2, M = 4, K = 20 (the bench's morphing workload): oracle at 2000 sampled (member, node).
    M, K, ny, nx, n_iter, tol = 4, 20, 4096, 4096, 20, 1e-5
    g = torch.Generator(device="cuda").manual_seed(9)
    # smooth fields at full size from a coarse seeded grid, upsampled on the device (inputs only)
    coarse_u = fields.smooth_members(41, M, K, 128, 128, ell=6.0)
    coarse_T = fields.smooth_mappings(42, K, 128, 128, amp=3.0, ell=6.0)
    up = torch.nn.Upsample(size=(ny, nx), mode="bilinear", align_corners=False)
    u = up(_dev(coarse_u)).contiguous()
    T = up(_dev(coarse_T)).contiguous()
    u_ref = u[:, 0].clone() + 0.1 * torch.randn((M, ny, nx), generator=g, device="cuda")
    ext = torch.empty((M + 2, K, ny, nx), dtype=torch.float32, device="cuda")
    ext[:2] = T
    _abi().fftenkf_morph_forward(u, u_ref, ext, M, K, ny, nx, n_iter, tol)
    out = torch.empty((M, K, ny, nx), dtype=torch.float32, device="cuda")
    _abi().fftenkf_morph_inverse(ext, u_ref, out, M, K, ny, nx)
    torch.cuda.synchronize()
    rng = np.random.default_rng(43)
    ks = rng.choice(np.array([0, 7, 13, 19]), 2000)
    ys = rng.integers(0, ny, 2000)
    xs = rng.integers(0, nx, 2000)
    for k in np.unique(ks):
        sel = ks == k
        Tk = T[:, k].cpu().numpy().astype(np.float64)
        qy, qx = morph.inverse_points_at(Tk, ys[sel], xs[sel], n_iter, tol)
        ek = ext[:, k].cpu().numpy().astype(np.float64)
        for j in range(M):
            uj = u[j, k].cpu().numpy().astype(np.float64)
            want = morph.interp_periodic(uj, qy, qx) - u_ref[j].cpu().numpy()[ys[sel], xs[sel]]
            got = ek[2 + j][ys[sel], xs[sel]]
            assert np.abs(got - want).max() <= ATOL
            # inverse: (u_ref + r) at p + T(p), r taken from the library's forward output
            f = u_ref[j].cpu().numpy().astype(np.float64) + ek[2 + j]
            want_i = morph.interp_periodic(f, ys[sel] + Tk[1][ys[sel], xs[sel]], xs[sel] + Tk[0][ys[sel], xs[sel]])
            got_i = out[j, k].cpu().numpy()[ys[sel], xs[sel]]
            assert np.abs(got_i - want_i).max() <= ATOL


def test_rejects_bad_arguments():
    abi = _abi()
    x = torch.zeros((3, 2, 8, 8), dtype=torch.float32, device="cuda")
    y = torch.zeros((1, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(abi.FftEnkfError) as e:
        abi.fftenkf_morph_forward(x[2:], y, x, 1, 2, 8, 8, 4)   # residual blocks alias u
    assert e.value.status == abi.FFTENKF_EINVAL
    with pytest.raises(abi.FftEnkfError):
        abi.fftenkf_morph_forward(x[:1], y, x, 1, 2, 8, 8, 2000)
    with pytest.raises(abi.FftEnkfError):
        abi.fftenkf_morph_forward(x[:1], y, x, 1, 2, 8, 8, 4, -1.0)
    with pytest.raises(abi.FftEnkfError):
        abi.fftenkf_morph_inverse(x, y, x, 1, 2, 8, 8)
    with pytest.raises(abi.FftEnkfError):
        abi.fftenkf_morph_reference(x, y, 3, 0, 8, 8)
