"""Parity at the benchmark's full sizes, on outputs the oracle can compute one
at a time (it builds the 80 hops of a sampled site from the links on the spot):

  * 8^4, FP64 apply of the whole lattice against the oracle's full apply;
  * 16^3x32 mixed-precision solves (FP32 and FP16 2-row hops, m0 = -0.05,
    links exp(i0.4H), Z2 source): the true residual b - D x at sampled sites;
  * 24^3x48 batched solve of the 12 spin-colour point sources (FP16 hops,
    m0 = 0): the residual at the source site, its neighbours and random sites;
  * 32^3x64 applies for every storage format and 4 right-hand sides, and the
    benchmark's own workload (FP32 full hops, 1 RHS, default launch shape) and
    its FP64 apply;
  * 12^4 fermion force: central finite differences of Re chi^dagger D psi in
    single link entries, evaluated over the 54 sites whose hops contain that
    link."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, synth

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)


def _site(L, x):
    x = [int(v) % L[m] for m, v in enumerate(x)]
    return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))


def _coords(L, s):
    out = []
    for m in range(4):
        out.append(s % L[m])
        s //= L[m]
    return out


def test_fp64_apply_8x8x8x8_whole_lattice(gpu):
    L = (8, 8, 8, 8)
    U = synth.random_su3_links(L, 0.3, 1012)
    psi = synth.gaussian_spinor(L, 1, 1013)[0]
    W = oracle.build_hops(L, U)
    ref = oracle.apply(L, AP, W, 0.0, psi)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu))
    x = torch.as_tensor(psi[None], device=gpu)
    out = op.apply(x, 0.0)
    for _ in range(9):  # ten applies, as the workload times them
        op.apply(x, 0.0, out=out)
    got = out.cpu().numpy()[0]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def _residual_sites(L, U, m0, x, b, sites):
    return b[sites] - oracle.apply_sites(L, AP, U, m0, x, sites)


@pytest.mark.parametrize("mode", [1, 2])
def test_mixed_solves_16x16x16x32(gpu, mode):
    L = (16, 16, 16, 32)
    U = synth.random_su3_links(L, 0.4, 1014)
    b = synth.z2_spinor(L, 1, 1015)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="2row")
    op.store_hops("f16", "2row")
    x, info = op.solve(torch.as_tensor(b, device=gpu), m0=-0.05, tol=1e-10, maxit=20000, mode=mode)
    assert info[0]["status"] == "BRI_OK" and info[0]["true_resid"] <= 1e-10, info
    V = synth.volume(L)
    sites = np.concatenate([[0, V - 1], np.random.default_rng(5).integers(0, V, 14)])
    r = _residual_sites(L, U, -0.05, x.cpu().numpy()[0], b[0], sites)
    # every component of r is bounded by ||r|| <= 1e-10 ||b||
    assert np.abs(r).max() <= 1e-10 * np.linalg.norm(b[0])


def test_batched_point_sources_24x24x24x48(gpu):
    L = (24, 24, 24, 48)
    V = synth.volume(L)
    U = synth.random_su3_links_torch(L, 0.35, 1016, device=gpu)
    op = Brillouin(L, AP)
    op.build_hops(U, prec="f16", comp="2row")
    x0 = int(np.random.default_rng(1017).integers(0, V))
    b = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device=gpu)
    for s_ in range(4):
        for c in range(3):
            b[3 * s_ + c, x0, s_, c] = 1.0
    x, info = op.solve(b, m0=0.0, tol=1e-10, maxit=20000, mode=3)
    assert all(i["status"] == "BRI_OK" and i["true_resid"] <= 1e-10 for i in info), info
    c0 = _coords(L, x0)
    sites = [x0] + [_site(L, [c0[m] + (1 if m == mu else 0) * sg for m in range(4)])
                    for mu in range(4) for sg in (1, -1)]
    sites = np.array(sites + list(np.random.default_rng(1018).integers(0, V, 4)))
    Uh = U.cpu().numpy()
    for r in (0, 5, 11):
        xr = x[r].cpu().numpy()
        br = b[r].cpu().numpy()
        res = _residual_sites(L, Uh, 0.0, xr, br, sites)
        assert np.abs(res).max() <= 1e-10 * np.linalg.norm(br)
    del op, U, x, b
    torch.cuda.empty_cache()


def test_storage_formats_and_rhs_32x32x32x64(gpu):
    L = (32, 32, 32, 64)
    V = synth.volume(L)
    U = synth.random_su3_links_torch(L, 0.3, 1015, device=gpu)
    psi = synth.gaussian_spinor_torch(L, 4, 1019, device=gpu).to(torch.complex64)
    op = Brillouin(L, AP)
    op.build_hops(U, prec="f32", comp="2row")
    sites = np.concatenate([[0, V - 1, 32 * 32 * 32 - 1], np.random.default_rng(7).integers(0, V, 5)])
    Uh = U.cpu().numpy()
    refs = [oracle.apply_sites(L, AP, Uh, 0.0, psi[r].cpu().numpy().astype(np.complex128), sites) for r in range(4)]
    # per-element bounds relative to max |ref| over the sampled sites, one per
    # (precision, link format): the lossy formats carry their own error
    for prec, comp, tol in (("f32", "2row", 1e-6), ("f32", "8param", 5e-5), ("f16", "full", 3e-4),
                            ("f16", "2row", 3e-4), ("f16", "8param", 1e-2)):
        op.store_hops(prec, comp)
        out = op.apply(psi, 0.0, prec=prec).cpu().numpy()
        for r in range(4):
            got = out[r][sites]
            err = np.abs(got - refs[r]).max() / np.abs(refs[r]).max()
            assert err <= tol, (prec, comp, r, err)
    del op, U, psi
    torch.cuda.empty_cache()


def test_benchmark_workload_32x32x32x64(gpu):
    """The benchmark's own workload and launch: links exp(i0.3H) (seed 1015),
    Gaussian FP32 spinor (seed 1115), FP32 full hops at the default launch
    shape, ten applies into the same output as the timed loop does; then the
    FP64 apply of the same field.  Sampled sites against the oracle."""
    L = (32, 32, 32, 64)
    V = synth.volume(L)
    U = synth.random_su3_links_torch(L, 0.3, 1015, device=gpu)
    x = synth.gaussian_spinor_torch(L, 1, 1115, device=gpu, dtype=torch.complex64)
    op = Brillouin(L, AP)
    op.build_hops(U, prec="f32", comp="full")
    out = torch.empty_like(x)
    for _ in range(10):
        op.apply(x, 0.0, prec="f32", out=out)
    sites = np.concatenate([[0, 31, 32 * 32 - 1, V // 2, V - 1], np.random.default_rng(11).integers(0, V, 7)])
    Uh = U.cpu().numpy()
    psi = x[0].cpu().numpy().astype(np.complex128)
    ref = oracle.apply_sites(L, AP, Uh, 0.0, psi, sites)
    got = out[0].cpu().numpy()[sites]
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
    del out
    x64 = x.to(torch.complex128)  # the FP64 fields stay next to the FP32 ones
    got64 = op.apply(x64, 0.0).cpu().numpy()[0][sites]
    assert np.abs(got64 - ref).max() <= 1e-13 * np.abs(ref).max()
    del op, U, x, x64
    torch.cuda.empty_cache()


def test_force_12x12x12x12_finite_differences(gpu):
    L = (12, 12, 12, 12)
    U = synth.random_su3_links(L, 0.3, 1020)
    chi, psi = synth.gaussian_spinor(L, 2, 1021)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu))
    dU = op.force(torch.as_tensor(chi, device=gpu), torch.as_tensor(psi, device=gpu)).cpu().numpy()
    rng = np.random.default_rng(1022)
    eps = 1e-5
    for _ in range(3):
        x0 = int(rng.integers(0, synth.volume(L)))
        mu = int(rng.integers(0, 4))
        a, bb = (int(v) for v in rng.integers(0, 3, 2))
        c0 = _coords(L, x0)
        # sites whose hops can contain the link (x0, mu): y_mu in {x0_mu, x0_mu + 1},
        # y_nu within one step of x0_nu
        sites = []
        for d in np.ndindex(2, 3, 3, 3):
            off = [0, 0, 0, 0]
            rest = [nu for nu in range(4) if nu != mu]
            off[mu] = d[0]
            for k, nu in enumerate(rest):
                off[nu] = d[k + 1] - 1
            sites.append(_site(L, [c0[m] + off[m] for m in range(4)]))
        sites = np.array(sorted(set(sites)))
        grad = 0
        for part, unit in ((0, 1.0), (1, 1j)):
            f = []
            for sg in (1, -1):
                Up = U.copy()
                Up[x0, mu, a, bb] += sg * eps * unit
                f.append(np.real(np.vdot(chi[sites], oracle.apply_sites(L, AP, Up, 0.0, psi, sites))))
            grad = grad + (1 if part == 0 else 1j) * (f[0] - f[1]) / (2 * eps)
        assert abs(dU[x0, mu, a, bb] - grad) <= 1e-7 * max(abs(grad), 1e-3), (dU[x0, mu, a, bb], grad)


def test_tensor_core_and_fp16_spinors_32x32x32x64(gpu):
    """32^3 x 64 at sampled sites: the tensor-core form with 12 right-hand
    sides (FP16 full fields, one warp pass) and the FP16-spinor apply (FP16
    2-row fields), each against the oracle built from the links at the sampled
    sites (bounds as in the small-lattice tests)."""
    L = (32, 32, 32, 64)
    V = synth.volume(L)
    U = synth.random_su3_links_torch(L, 0.3, 1015, device=gpu)
    psi = synth.gaussian_spinor_torch(L, 12, 1021, device=gpu).to(torch.complex64)
    op = Brillouin(L, AP)
    op.build_hops(U, prec="f16", comp="full")
    op.set_threads("f16", 12, 16384)
    out = op.apply(psi, 0.02, prec="f16").cpu().numpy()
    sites = np.concatenate([[0, V - 1, 31, 32 * 32 * 32 - 1], np.random.default_rng(13).integers(0, V, 4)])
    Uh = U.cpu().numpy()
    for r in (0, 5, 11):
        ref = oracle.apply_sites(L, AP, Uh, 0.02, psi[r].cpu().numpy().astype(np.complex128), sites)
        err = np.abs(out[r][sites] - ref).max() / np.abs(ref).max()
        assert err <= 5e-4, (r, err)
    del out
    op.store_hops("f16", "2row")
    xh = op.to_h16(psi[:1].contiguous())
    dec = op.from_h16(xh, torch.complex128)[0].cpu().numpy()
    got = op.from_h16(op.apply(xh, 0.02, prec="f16h"), torch.complex128)[0].cpu().numpy()[sites]
    ref = oracle.apply_sites(L, AP, Uh, 0.02, dec, sites)
    assert np.abs(got - ref).max() <= 6e-4 * np.abs(ref).max()
    del op, U, psi
    torch.cuda.empty_cache()
