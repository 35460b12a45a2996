"""FP16 spinors with one FP32 scale per site (prec "f16h", reading A14 of the
spinor precision: IEEE binary16, round to nearest, power-of-two scale per
site): the conversion matches its definition, and the apply on FP16 hopping
fields and FP16 spinors matches the oracle applied to the decoded input,
element by element, to the FP16 bounds stated here."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, BriError, synth

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)
# per-element bound (of max |ref|): FP16 links (3e-4, 8-parameter 1e-2) plus
# the rounding of the output to 11 bits of its site's largest component
TOL = {"full": 6e-4, "2row": 6e-4, "8param": 1.2e-2}


def _rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("L,nrhs", [((3, 3, 3, 3), 3), ((4, 3, 5, 4), 2)])
def test_h16_conversion_follows_its_definition(gpu, L, nrhs):
    """scale = the power of two 2^e with the site's max |component| in
    [2^(e-1), 2^e); entries = fp16(v / scale) rounded to nearest."""
    op = Brillouin(L, AP)
    psi = synth.gaussian_spinor(L, nrhs, 11).astype(np.complex64)
    psi[0, 5] *= 1e-20  # a tiny site and a zero site keep their own scales
    psi[-1, 7] = 0
    x = torch.as_tensor(psi, device=gpu)
    buf = op.to_h16(x)
    assert buf.shape == (nrhs, op.h16_field_bytes())
    V = synth.volume(L)
    raw = buf.cpu().numpy()
    for r in range(nrhs):
        halves = raw[r, :48 * V].view(np.float16).reshape(V, 12, 2).astype(np.float64)
        scales = raw[r, 48 * V:52 * V].view(np.float32).astype(np.float64)
        comps = np.stack([psi[r].real, psi[r].imag], -1).reshape(V, 24).astype(np.float64)
        m = np.abs(comps).max(1)
        want_scale = np.where(m > 0, np.ldexp(1.0, np.frexp(m)[1]), 1.0)
        assert np.array_equal(scales, want_scale)
        want = (comps / want_scale[:, None]).astype(np.float16).astype(np.float64)
        assert np.array_equal(halves.reshape(V, 24), want)
    back = op.from_h16(buf).cpu().numpy()
    for r in range(nrhs):
        # each real component within half an FP16 ulp of (-1, 1), times the site's scale
        comps = np.stack([psi[r].real, psi[r].imag], -1).reshape(V, 24).astype(np.float64)
        got = np.stack([back[r].real, back[r].imag], -1).reshape(V, 24).astype(np.float64)
        m = np.abs(comps).max(1)
        scale = np.where(m > 0, np.ldexp(1.0, np.frexp(m)[1]), 1.0)
        assert np.all(np.abs(got - comps) <= 2.0 ** -12 * scale[:, None])


@pytest.mark.parametrize("comp", ["full", "2row", "8param"])
@pytest.mark.parametrize("L,nrhs", [((3, 3, 3, 3), 3), ((3, 5, 4, 6), 2), ((4, 4, 4, 6), 1), ((32, 3, 4, 4), 2)])
def test_h16_apply_matches_oracle(gpu, comp, L, nrhs):
    """x extent 32: the bulk-copy line kernel with the FP16 spinor lines
    staged (halves and scales); otherwise the pair loop."""
    U = synth.random_su3_links(L, 0.4, 40 + sum(L))
    psi = synth.gaussian_spinor(L, nrhs, 41 + sum(L)).astype(np.complex64)
    W = oracle.build_hops(L, U)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f16", comp=comp)
    xh = op.to_h16(torch.as_tensor(psi, device=gpu))
    dec = op.from_h16(xh, torch.complex128).cpu().numpy()  # the input as stored
    outs = [op.from_h16(op.apply(xh, 0.03, prec="f16h"), torch.complex128).cpu().numpy(),
            op.from_h16(op.apply(xh, 0.03, dagger=True, prec="f16h"), torch.complex128).cpu().numpy(),
            op.from_h16(op.overlap_kernel(xh, 1.0, prec="f16h"), torch.complex128).cpu().numpy()]
    for r in range(nrhs):
        refs = [oracle.apply(L, AP, W, 0.03, dec[r]), oracle.apply(L, AP, W, 0.03, dec[r], dagger=True),
                oracle.overlap_kernel(L, AP, W, 0.0, 1.0, dec[r])]
        for o, ref, what in zip(outs, refs, ("D", "Ddag", "H")):
            e = _rel_max(o[r], ref)
            assert e < TOL[comp], (what, r, e)


def test_h16_requires_fp16_fields_and_checks_sizes(gpu):
    L = (3, 3, 3, 4)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(synth.random_su3_links(L, 0.3, 5), device=gpu), prec="f32")
    xh = op.to_h16(synth.gaussian_spinor_torch(L, 1, 6, device=gpu, dtype=torch.complex64))
    with pytest.raises(BriError, match="BRI_ESTATE"):
        op.apply(xh, 0.0, prec="f16h")  # no FP16 fields stored
    op.store_hops("f16", "2row")
    out = op.apply(xh, 0.0, prec="f16h")
    assert out.shape == xh.shape
    with pytest.raises(ValueError):
        op.apply(xh[:, :-16].contiguous(), 0.0, prec="f16h")
