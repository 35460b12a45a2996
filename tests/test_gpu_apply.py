"""GPU stencil apply (Eq. def_pref, class form of Sec. 8) against the CPU
oracle, element by element (max |gpu - ref| / max |ref|): FP64 to 1e-13,
FP32 full and 2-row fields to 1e-6, for D, D^dagger and the overlap kernel
gamma_5 (D - rho).  The lossy storage formats carry their own bounds
(``TOL_MAX``): FP16 fields round every link entry to 11 bits, and the
8-parameter form reconstructs |U00| and |U20| through square roots and
divides by 1 - |U00|^2, both ill-conditioned near diagonal links, so its
FP32 error is a property of the format, not of the arithmetic."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, BriError, synth
from paper_1012_3615_gb300.core import WEIGHTS

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)
PER = (1, 1, 1, 1)

CASES = [((4, 4, 4, 4), AP), ((3, 5, 4, 6), AP), ((4, 3, 3, 4), PER), ((3, 3, 3, 3), AP)]
# extents that are multiples of the shared-memory tile (8, 4, 2, 2), where the
# tiled kernel can be selected
TILED = [((8, 4, 4, 4), AP), ((16, 8, 6, 4), PER)]


def _setup(L, bc, seed, nrhs=2, eps=0.4):
    U = synth.random_su3_links(L, eps, seed)
    psi = synth.gaussian_spinor(L, nrhs, seed + 1)
    W = oracle.build_hops(L, U)
    return U, psi, W


def _rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# per-element bounds (relative to max |ref|) per (precision, link format)
TOL_MAX = {("f32", "full"): 1e-6, ("f32", "2row"): 1e-6, ("f32", "8param"): 5e-5,
           ("f16", "full"): 3e-4, ("f16", "2row"): 3e-4, ("f16", "8param"): 1e-2}


def _check(out, ref, tol, what=""):
    """element-wise parity; the relative 2-norm is reported alongside"""
    e = _rel_max(out, ref)
    assert e < tol, (what, e, _rel_l2(out, ref))


@pytest.mark.parametrize("L,bc", CASES)
def test_fp64_apply_dagger_overlap(gpu, L, bc):
    U, psi, W = _setup(L, bc, sum(L))
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu))
    x = torch.as_tensor(psi, device=gpu)
    m0 = -0.07
    out = op.apply(x, m0=m0).cpu().numpy()
    outd = op.apply(x, m0=m0, dagger=True).cpu().numpy()
    outh = op.overlap_kernel(x, rho=1.0).cpu().numpy()
    for r in range(psi.shape[0]):
        assert _rel_max(out[r], oracle.apply(L, bc, W, m0, psi[r])) < 1e-13
        assert _rel_max(outd[r], oracle.apply(L, bc, W, m0, psi[r], dagger=True)) < 1e-13
        assert _rel_max(outh[r], oracle.overlap_kernel(L, bc, W, 0.0, 1.0, psi[r])) < 1e-13


@pytest.mark.parametrize("comp", ["full", "2row", "8param"])
@pytest.mark.parametrize("L,bc", CASES[:2] + TILED)
def test_fp32_apply(gpu, L, bc, comp):
    tol = TOL_MAX[("f32", comp)]
    U, psi, W = _setup(L, bc, 10 + sum(L))
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp=comp)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    for dag in (False, True):
        out = op.apply(x, m0=0.02, dagger=dag, prec="f32").cpu().numpy()
        for r in range(psi.shape[0]):
            ref = oracle.apply(L, bc, W, 0.02, psi[r], dagger=dag)
            _check(out[r], ref, tol, (dag, r))
    outh = op.overlap_kernel(x, rho=1.0, prec="f32").cpu().numpy()
    _check(outh[0], oracle.overlap_kernel(L, bc, W, 0.0, 1.0, psi[0]), tol, "overlap kernel")


@pytest.mark.parametrize("comp", ["full", "2row", "8param"])
def test_fp16_links_apply(gpu, comp):
    tol = TOL_MAX[("f16", comp)]
    L, bc = (4, 4, 4, 6), AP
    U, psi, W = _setup(L, bc, 21)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f16", comp=comp)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    out = op.apply(x, m0=0.0, prec="f16").cpu().numpy()
    for r in range(psi.shape[0]):
        _check(out[r], oracle.apply(L, bc, W, 0.0, psi[r]), tol, r)


@pytest.mark.parametrize("prec,comp", [("f32", "full"), ("f32", "2row"), ("f16", "2row")])
def test_tiled_kernel_equals_plain_kernel(gpu, prec, comp):
    """The shared-memory tiled kernel performs the same arithmetic in the same
    order as the plain one: results are bitwise equal, for every mode."""
    L, bc = (16, 8, 6, 4), AP
    U = synth.random_su3_links(L, 0.4, 31)
    psi = synth.gaussian_spinor(L, 3, 32).astype(np.complex64)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp=comp)
    x = torch.as_tensor(psi, device=gpu)
    op.set_threads(prec, 3, 0)  # tiled kernel
    tiled = [op.apply(x, 0.1, prec=prec), op.apply(x, 0.1, dagger=True, prec=prec), op.overlap_kernel(x, 1.0, prec=prec)]
    op.set_threads(prec, 3, 128)
    plain = [op.apply(x, 0.1, prec=prec), op.apply(x, 0.1, dagger=True, prec=prec), op.overlap_kernel(x, 1.0, prec=prec)]
    for a, b in zip(tiled, plain):
        assert torch.equal(a, b)


@pytest.mark.parametrize("prec,comp", [("f32", "full"), ("f32", "2row"), ("f32", "8param"), ("f16", "full"),
                                       ("f16", "2row"), ("f16", "8param")])
def test_kernel_variants_agree(gpu, prec, comp):
    """Every launch shape of the FP32-arithmetic stencil (plain kernel at several
    block sizes, register link prefetch, cp.async link prefetch, fewer-register
    form, (d, -d) pair-combined form, bulk-copy link pipeline) computes the
    same result to FP32 rounding."""
    L, bc = (6, 5, 4, 8), AP
    U = synth.random_su3_links(L, 0.4, 41)
    psi = synth.gaussian_spinor(L, 2, 42).astype(np.complex64)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp=comp)
    x = torch.as_tensor(psi, device=gpu)
    outs = []
    for shape in (128, 64, 256, 2048 + 128, 4096 + 64, 4096 + 128, 4096 + 256, 8192 + 128, 8192 + 256,
                  5 * 2048 + 64, 5 * 2048 + 128, 5 * 2048 + 256, 6 * 2048 + 128, 7 * 2048 + 128, 9 * 2048 + 128,
                  10 * 2048 + 64, 10 * 2048 + 128, 10 * 2048 + 256, 11 * 2048 + 32):
        op.set_threads(prec, 2, shape)
        outs.append((shape, op.apply(x, -0.2, dagger=True, prec=prec)))
    for shape, o in outs[1:]:
        err = (torch.abs(o - outs[0][1]).max() / torch.abs(outs[0][1]).max()).item()
        assert err < 1e-6, (shape, err)


@pytest.mark.parametrize("prec,comp", [("f32", "full"), ("f32", "2row"), ("f16", "full"), ("f16", "2row")])
@pytest.mark.parametrize("L,bc", [((3, 5, 4, 6), AP), ((4, 4, 4, 4), PER), ((8, 4, 4, 8), AP)])
def test_pair_kernel_matches_oracle(gpu, prec, comp, L, bc):
    """The site-pair kernel (two sites i, i + V/2 per thread, pair-interleaved
    links) against the oracle for D, D^dagger and the overlap kernel."""
    tol = TOL_MAX[(prec, comp)]
    U, psi, W = _setup(L, bc, 50 + sum(L))
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp=comp)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    for shape in (6144 + 64, 6144 + 128):
        op.set_threads(prec, 2, shape)
        out = op.apply(x, m0=0.05, prec=prec).cpu().numpy()
        outd = op.apply(x, m0=0.05, dagger=True, prec=prec).cpu().numpy()
        outh = op.overlap_kernel(x, rho=1.0, prec=prec).cpu().numpy()
        for r in range(psi.shape[0]):
            _check(out[r], oracle.apply(L, bc, W, 0.05, psi[r]), tol, (shape, "D"))
            _check(outd[r], oracle.apply(L, bc, W, 0.05, psi[r], dagger=True), tol, (shape, "Ddag"))
            _check(outh[r], oracle.overlap_kernel(L, bc, W, 0.0, 1.0, psi[r]), tol, (shape, "H"))


@pytest.mark.parametrize("prec,comp", [("f32", "full"), ("f32", "2row"), ("f32", "8param"), ("f16", "2row")])
@pytest.mark.parametrize("L,bc", [((3, 5, 4, 6), AP), ((4, 4, 4, 4), PER)])
def test_pair_combined_body_matches_oracle(gpu, prec, comp, L, bc):
    """The loops that combine the hops d and -d before the gamma terms (launch
    variants 5-7, 9, 10) against the oracle for D, D^dagger and the overlap
    kernel, with the Brillouin and the Wilson weights."""
    tol = TOL_MAX[(prec, comp)]
    U, psi, W = _setup(L, bc, 60 + sum(L))
    for name in ("brillouin", "wilson"):
        lam, rho = WEIGHTS[name]
        op = Brillouin(L, bc)
        op.set_weights(lam, rho)
        op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp=comp)
        x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
        oracle.set_weights(lam, rho)
        try:
            ref = [(oracle.apply(L, bc, W, 0.05, psi[r]), oracle.apply(L, bc, W, 0.05, psi[r], dagger=True),
                    oracle.overlap_kernel(L, bc, W, 0.0, 1.0, psi[r])) for r in range(psi.shape[0])]
        finally:
            oracle.reset_weights()
        for shape in (5 * 2048 + 64, 5 * 2048 + 128, 6 * 2048 + 128, 7 * 2048 + 128, 9 * 2048 + 128,
                      10 * 2048 + 128):
            op.set_threads(prec, 2, shape)
            out = op.apply(x, m0=0.05, prec=prec).cpu().numpy()
            outd = op.apply(x, m0=0.05, dagger=True, prec=prec).cpu().numpy()
            outh = op.overlap_kernel(x, rho=1.0, prec=prec).cpu().numpy()
            for r in range(psi.shape[0]):
                _check(out[r], ref[r][0], tol, (shape, name, "D"))
                _check(outd[r], ref[r][1], tol, (shape, name, "Ddag"))
                _check(outh[r], ref[r][2], tol, (shape, name, "H"))


@pytest.mark.parametrize("prec,comp", [("f32", "full"), ("f32", "2row"), ("f32", "8param"), ("f16", "full"),
                                       ("f16", "2row"), ("f16", "8param")])
@pytest.mark.parametrize("L,bc", [((32, 3, 4, 4), AP), ((16, 4, 3, 4), PER), ((64, 3, 3, 3), AP),
                                  ((3, 5, 4, 6), AP)])
def test_bulk_copy_kernel_matches_oracle(gpu, prec, comp, L, bc):
    """The bulk-copy link pipeline (launch variant 10) against the oracle for
    D, D^dagger and the overlap kernel, at 32, 64 and 128 threads.  The x
    extents cover its cases: 32 (a warp is one x line, every x - d in one
    staged block, three stages; at 32 threads the one-warp-per-block line
    kernel), 16 and 64 (x - d in two blocks, two stages of three runs), 3 (a
    warp spans many x lines: lanes outside the staged blocks load their
    reversed links from global memory; 360 sites, a ragged last warp).
    Variant 11 (x extent 32: links and neighbour spinor lines staged, two or
    three link stages) falls back to variant 10 at the other extents."""
    tol = TOL_MAX[(prec, comp)]
    U, psi, W = _setup(L, bc, 70 + sum(L))
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp=comp)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    ref = [(oracle.apply(L, bc, W, -0.1, psi[r]), oracle.apply(L, bc, W, -0.1, psi[r], dagger=True),
            oracle.overlap_kernel(L, bc, W, 0.0, 1.0, psi[r])) for r in range(psi.shape[0])]
    for shape in (10 * 2048 + 32, 10 * 2048 + 64, 10 * 2048 + 128, 11 * 2048 + 32, 11 * 2048 + 64):
        op.set_threads(prec, 2, shape)
        out = op.apply(x, m0=-0.1, prec=prec).cpu().numpy()
        outd = op.apply(x, m0=-0.1, dagger=True, prec=prec).cpu().numpy()
        outh = op.overlap_kernel(x, rho=1.0, prec=prec).cpu().numpy()
        for r in range(psi.shape[0]):
            _check(out[r], ref[r][0], tol, (shape, "D"))
            _check(outd[r], ref[r][1], tol, (shape, "Ddag"))
            _check(outh[r], ref[r][2], tol, (shape, "H"))


@pytest.mark.parametrize("name", ["wilson", "hypercube"])
@pytest.mark.parametrize("prec,comp", [("f32", "full"), ("f16", "2row")])
def test_bulk_copy_kernel_other_weights(gpu, name, prec, comp):
    """The line kernel (launch variant 11, x extent 32) with the Wilson and the
    hypercube columns of the weight table: the hop list then holds other
    groups of equal (d_y, d_z, d_t) (Wilson: four single-hop groups), which the
    kernel's spinor-line staging follows."""
    L, bc = (32, 3, 3, 4), AP
    tol = TOL_MAX[(prec, comp)]
    U, psi, W = _setup(L, bc, 90)
    lam, rho = WEIGHTS[name]
    op = Brillouin(L, bc)
    op.set_weights(lam, rho)
    op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp=comp)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    oracle.set_weights(lam, rho)
    try:
        ref = [(oracle.apply(L, bc, W, 0.05, psi[r]), oracle.apply(L, bc, W, 0.05, psi[r], dagger=True))
               for r in range(psi.shape[0])]
    finally:
        oracle.reset_weights()
    for shape in (11 * 2048 + 32, 11 * 2048 + 64):
        op.set_threads(prec, 2, shape)
        out = op.apply(x, m0=0.05, prec=prec).cpu().numpy()
        outd = op.apply(x, m0=0.05, dagger=True, prec=prec).cpu().numpy()
        for r in range(psi.shape[0]):
            _check(out[r], ref[r][0], tol, (shape, name, "D"))
            _check(outd[r], ref[r][1], tol, (shape, name, "Ddag"))


def test_multi_rhs_equals_single(gpu):
    L, bc = (4, 3, 5, 4), AP
    U = synth.random_su3_links(L, 0.3, 5)
    psi = synth.gaussian_spinor(L, 24, 6)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="2row")
    for prec, dt in (("f64", np.complex128), ("f32", np.complex64)):
        x = torch.as_tensor(psi.astype(dt), device=gpu)
        many = op.apply(x, 0.1, prec=prec)
        for r in (0, 7, 23):
            one = op.apply(x[r:r + 1].contiguous(), 0.1, prec=prec)
            assert torch.equal(many[r:r + 1], one)


def test_free_field_plane_wave_on_gpu(gpu):
    """U = 1: D acts on exp(i k.x) u as the momentum-space symbol built from
    the closed forms of Eq. def_4Dbri and App. C (no oracle involved)."""
    L, bc = (8, 8, 6, 12), AP
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(synth.unit_links(L), device=gpu))
    rng = np.random.default_rng(3)
    for _ in range(4):
        k = [2 * np.pi * rng.integers(0, L[m]) / L[m] for m in range(3)] + \
            [(2 * rng.integers(0, L[3]) + 1) * np.pi / L[3]]
        k = np.array(k)
        u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        psi = synth.plane_wave(L, k, u)
        out = op.apply(torch.as_tensor(psi, device=gpu), m0=0.3).cpu().numpy()
        M = (0.3 + 2 - 2 * np.prod(np.cos(k / 2) ** 2)) * np.eye(4, dtype=complex)
        for mu in range(4):
            M = M + 1j * np.sin(k[mu]) * np.prod([np.cos(k[nu]) + 2 for nu in range(4) if nu != mu]) / 27 \
                * oracle.gamma(mu)
        expect = synth.plane_wave(L, k, M @ u)
        assert _rel_max(out, expect) < 1e-13


def test_gauge_covariance_and_gamma5_hermiticity_on_gpu(gpu):
    L, bc = (6, 6, 6, 8), AP
    U = synth.random_su3_links(L, 0.4, 8)
    g = synth.gauge_transform(L, 9)
    x = synth.coordinates(L)
    Ug = np.empty_like(U)
    for mu in range(4):
        y = x.copy()
        y[:, mu] = (y[:, mu] + 1) % L[mu]
        yi = y[:, 0] + L[0] * (y[:, 1] + L[1] * (y[:, 2] + L[2] * y[:, 3]))
        Ug[:, mu] = g @ U[:, mu] @ g[yi].conj().transpose(0, 2, 1)
    psi, phi = synth.gaussian_spinor(L, 2, 10)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu))
    Dpsi = op.apply(torch.as_tensor(psi, device=gpu), -0.1).cpu().numpy()
    Ddphi = op.apply(torch.as_tensor(phi, device=gpu), -0.1, dagger=True).cpu().numpy()
    assert abs(np.vdot(phi, Dpsi) - np.vdot(Ddphi, psi)) < 1e-10 * abs(np.vdot(phi, Dpsi))
    op.build_hops(torch.as_tensor(Ug, device=gpu))
    gpsi = np.einsum("xab,xsb->xsa", g, psi)
    lhs = op.apply(torch.as_tensor(gpsi, device=gpu), -0.1).cpu().numpy()
    assert _rel_max(lhs, np.einsum("xab,xsb->xsa", g, Dpsi)) < 1e-12


def test_full_size_sampled_sites(gpu):
    """32^3 x 64 in the benchmark's launch configuration (FP32 full links,
    tuned block size) and in FP64: sampled output sites against the oracle,
    which builds the hops of each sampled site from U on the spot."""
    L, bc = (32, 32, 32, 64), AP
    U = synth.random_su3_links_torch(L, 0.3, 1015, device=gpu)
    psi = synth.gaussian_spinor_torch(L, 1, 1016, device=gpu)
    op = Brillouin(L, bc)
    op.build_hops(U, prec="f32", comp="full")
    out64 = op.apply(psi, 0.0, prec="f64")
    out32 = op.apply(psi.to(torch.complex64), 0.0, prec="f32")
    rng = np.random.default_rng(11)
    V = synth.volume(L)
    sites = np.concatenate([[0, V - 1, 31, V - 32 * 32 * 32], rng.integers(0, V, 6)])
    Uh = U.cpu().numpy()
    ph = psi[0].cpu().numpy()
    ref = oracle.apply_sites(L, bc, Uh, 0.0, ph, sites)
    g64 = out64[0].cpu().numpy()[sites]
    g32 = out32[0].cpu().numpy()[sites]
    assert _rel_max(g64, ref) < 1e-13
    _check(g32, ref, 1e-6, "32^3x64 FP32 sampled sites")
    del op
    torch.cuda.empty_cache()


def test_argument_errors(gpu):
    L = (3, 3, 3, 3)
    op = Brillouin(L, AP)
    x = torch.zeros((1, 81, 4, 3), dtype=torch.complex128, device=gpu)
    with pytest.raises(BriError, match="BRI_ESTATE"):
        op.apply(x)  # no hops yet
    op.build_hops(torch.as_tensor(synth.unit_links(L), device=gpu))
    with pytest.raises(BriError, match="BRI_ESTATE"):
        op.apply(x.to(torch.complex64), prec="f32")  # FP32 fields not stored
    with pytest.raises(BriError, match="BRI_EINVAL"):
        op.apply(x, out=x)  # in-place
    big = torch.zeros(81 * 12 + 1, dtype=torch.complex64, device=gpu)
    with pytest.raises(BriError, match="BRI_EINVAL"):
        op.apply(big[1:].view(1, 81, 4, 3), prec="f32")  # 8-byte offset: not 16-byte aligned
    with pytest.raises(BriError):
        Brillouin((2, 4, 4, 4))


@pytest.mark.parametrize("L", [(4, 3, 4, 3), (4, 4, 3, 6), (3, 4, 4, 12), (32, 3, 3, 8)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_apply_host_buffers_match_device_apply(gpu, L, prec):
    """bri_apply_host (slabs in t, copies overlapping the stencil) gives the
    device apply bit for bit, pinned or pageable, D and D^dagger, 2 RHS (x
    extent 32: the bulk-copy line kernel on whole-line site ranges)."""
    U = synth.random_su3_links(L, 0.4, 51)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32" if prec == "f32" else "f64", comp="full")
    psi = synth.gaussian_spinor(L, 2, 52)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    xd = torch.as_tensor(psi, device=gpu).to(dt).contiguous()
    for pinned in (True, False):
        xh = xd.cpu()
        if pinned:
            xh = xh.pin_memory()
        for dag in (False, True):
            want = op.apply(xd, 0.07, dagger=dag, prec=prec).cpu()
            got = op.apply_host(xh, 0.07, dagger=dag, prec=prec)
            torch.cuda.synchronize()
            assert torch.equal(got, want)


@pytest.mark.parametrize("L", [(3, 3, 3, 3), (32, 3, 3, 3)])
def test_many_right_hand_sides(gpu, L):
    """1000 right-hand sides in one launch (grid of site blocks, or x lines for
    the line kernel on an x extent of 32, times RHS): every RHS equals its own
    single apply."""
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(synth.random_su3_links(L, 0.5, 71), device=gpu), prec="f32")
    x = synth.gaussian_spinor_torch(L, 1000, 72, device=gpu).to(torch.complex64)
    many = op.apply(x, 0.2, prec="f32")
    for r in (0, 1, 499, 998, 999):
        assert torch.equal(many[r:r + 1], op.apply(x[r:r + 1].contiguous(), 0.2, prec="f32"))


def test_tuner_choice_is_correct_and_cached(gpu, tmp_path, monkeypatch):
    """bri_tune times its candidate launch shapes (the bulk-copy variants
    among them on an x extent of 32) and keeps the fastest; the apply with that
    shape matches the oracle, the choice is appended to BRI_TUNE_CACHE, and a
    new context reads it back, variant bits included."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("BRI_TUNE_CACHE", str(cache))
    L, bc = (32, 3, 4, 4), AP
    U, psi, W = _setup(L, bc, 95)
    op = Brillouin(L, bc)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="2row")
    op.tune("f32", 2)
    shape = op.threads("f32", 2)
    assert shape >= 0
    out = op.apply(torch.as_tensor(psi.astype(np.complex64), device=gpu), 0.05, prec="f32").cpu().numpy()
    for r in range(psi.shape[0]):
        _check(out[r], oracle.apply(L, bc, W, 0.05, psi[r]), TOL_MAX[("f32", "2row")], ("tuned", shape))
    assert cache.read_text().split()[-1] == str(shape)
    op2 = Brillouin(L, bc)
    op2.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="2row")
    assert op2.threads("f32", 2) == shape
    # a cached shape with the variant bits of the line kernel survives the reload
    cache.write_text(cache.read_text() + "dslash:32x3x4x4:p1:c1:n3 %d\n" % (11 * 2048 + 64))
    op3 = Brillouin(L, bc)
    op3.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="2row")
    assert op3.threads("f32", 3) == 11 * 2048 + 64
