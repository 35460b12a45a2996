"""Tensor-core multi-RHS apply (launch variant 16384: the class form of
Sec. 8 as one complex (15 x 240) x (240 x 4N) product per site on mma.sync,
FP16 operands, FP32 accumulation) against the oracle, element by element.

The operands are rounded to 11-bit mantissas (links times class weights,
spinors scaled per right-hand side by a power of two), so the bound is that of
FP16 operands: 5e-4 of max |ref| (the model of the rounding gives ~1e-4 for D
and 2e-4 for gamma_5 (D - rho), whose diagonal is smaller)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1012_3615_gb300 import Brillouin, synth
from paper_1012_3615_gb300.core import WEIGHTS

pytestmark = pytest.mark.gpu
AP = (1, 1, 1, -1)
TC = 16384
TOL = 5e-4


def _rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec", ["f16", "f32"])
@pytest.mark.parametrize("L,nrhs", [((4, 4, 4, 4), 1), ((3, 5, 4, 6), 2), ((3, 5, 4, 6), 5), ((4, 3, 5, 4), 12),
                                    ((3, 3, 3, 5), 13), ((3, 4, 3, 3), 24), ((4, 6, 4, 4), 13), ((6, 4, 4, 4), 8)])
def test_tc_apply_matches_oracle(gpu, prec, L, nrhs):
    U = synth.random_su3_links(L, 0.4, 80 + nrhs)
    psi = synth.gaussian_spinor(L, nrhs, 81 + nrhs)
    W = oracle.build_hops(L, U)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec=prec, comp="full")
    op.set_threads(prec, nrhs, TC)
    x = torch.as_tensor(psi.astype(np.complex64), device=gpu)
    n0 = op.kernel_launches()
    out = op.apply(x, m0=0.03, prec=prec).cpu().numpy()
    assert op.kernel_launches() - n0 == 3  # per-RHS scale, FP16 copy of the spinors, stencil
    outd = op.apply(x, m0=0.03, dagger=True, prec=prec).cpu().numpy()
    outh = op.overlap_kernel(x, rho=1.0, prec=prec).cpu().numpy()
    for r in range(nrhs):
        psr = psi[r].astype(np.complex64).astype(np.complex128)
        assert _rel_max(out[r], oracle.apply(L, AP, W, 0.03, psr)) < TOL, ("D", r)
        assert _rel_max(outd[r], oracle.apply(L, AP, W, 0.03, psr, dagger=True)) < TOL, ("Ddag", r)
        assert _rel_max(outh[r], oracle.overlap_kernel(L, AP, W, 0.0, 1.0, psr)) < TOL, ("H", r)


def test_tc_apply_scale_invariance_and_zero_fields(gpu):
    """Right-hand sides of very different magnitude (1e-30 .. 1e20) in one
    launch, and an all-zero one: the per-RHS power-of-two scale keeps every
    operand inside the FP16 range, so each result has the same relative error."""
    L = (4, 3, 4, 4)
    U = synth.random_su3_links(L, 0.4, 91)
    psi = synth.gaussian_spinor(L, 4, 92)
    scales = [1e-30, 1.0, 1e20, 0.0]
    psi = psi * np.array(scales)[:, None, None, None]
    W = oracle.build_hops(L, U)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f16", comp="full")
    op.set_threads("f16", 4, TC)
    out = op.apply(torch.as_tensor(psi.astype(np.complex64), device=gpu), m0=0.0, prec="f16").cpu().numpy()
    for r in range(3):
        psr = psi[r].astype(np.complex64).astype(np.complex128)
        assert _rel_max(out[r], oracle.apply(L, AP, W, 0.0, psr)) < TOL, r
    assert np.all(out[3] == 0)


@pytest.mark.parametrize("name", ["wilson", "hypercube"])
def test_tc_apply_other_weight_columns(gpu, oracle_weights, name):
    """Other members of the class (Tab. rholambda): the Wilson column has 4 hop
    pairs (one group of 8 hops), the hypercube one all 40."""
    lam, rho = WEIGHTS[name]
    oracle_weights(lam, rho)
    L, nrhs = (4, 3, 5, 4), 6
    U = synth.random_su3_links(L, 0.4, 93)
    psi = synth.gaussian_spinor(L, nrhs, 94)
    W = oracle.build_hops(L, U)
    op = Brillouin(L, AP)
    op.set_weights(lam, rho)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f16", comp="full")
    op.set_threads("f16", nrhs, TC)
    out = op.apply(torch.as_tensor(psi.astype(np.complex64), device=gpu), m0=0.1, prec="f16").cpu().numpy()
    for r in range(nrhs):
        psr = psi[r].astype(np.complex64).astype(np.complex128)
        assert _rel_max(out[r], oracle.apply(L, AP, W, 0.1, psr)) < TOL, r


def test_tc_falls_back_for_compressed_fields(gpu):
    """2-row fields: variant 16384 runs the untuned FP32-arithmetic stencil."""
    L = (4, 4, 3, 4)
    U = synth.random_su3_links(L, 0.4, 95)
    psi = synth.gaussian_spinor(L, 3, 96).astype(np.complex64)
    op = Brillouin(L, AP)
    op.build_hops(torch.as_tensor(U, device=gpu), prec="f32", comp="2row")
    x = torch.as_tensor(psi, device=gpu)
    ref = op.apply(x, 0.0, prec="f32")
    op.set_threads("f32", 3, TC)
    assert torch.equal(op.apply(x, 0.0, prec="f32"), ref)
