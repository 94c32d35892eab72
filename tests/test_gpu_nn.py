"""GPU parity of the learned gauge-covariant layer (``oracle.nn``).

Forward FP32 against the FP64 oracle within 1e-5 (sums of at most 72 FP32
products per component); FP16 hidden channels and weights within 5e-3 (FP16
keeps 11 significant bits); the two-layer network with the Wilson weights in
layer 2 reproduces D_W at c_sw = 0; loss and Wirtinger gradient within 1e-4;
training pairs e = (1 - B D) e0, r = D e against the oracle's K-cycle with a
fixed coarse step count; Adam lowers the loss; FGMRES with the learned stage
(and with its SAP stand-in) reaches 1e-10.
"""
import numpy as np
import pytest

import inputs
from oracle import nn
from oracle.dirac import Operator
from oracle.amg import TwoLevel, AMGParams

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1611_01034_gb300 as tm  # noqa: E402
from tests.gpu_helpers import GPU, rel  # noqa: E402

F32, F16 = tm.TM_F32, tm.TM_F16


def _weights(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    w = scale * (rng.standard_normal(2304) + 1j * rng.standard_normal(2304))
    return nn.unpack_weights(w)


def _fields(L, n, seed):
    rng = np.random.default_rng(seed)
    s = (n,) + tuple(L) + (4, 3)
    return rng.standard_normal(s) + 1j * rng.standard_normal(s)


# aggregate / SAP block per lattice (6x6x4x10: 1440 sites, not a multiple of the
# 64-site gradient tile or the 128-thread layer CTA)
AGG = {(4, 4, 4, 4): (2, 2, 2, 2), (6, 6, 4, 10): (3, 3, 2, 5), (4, 4, 4, 8): (2, 2, 2, 2),
       (8, 4, 4, 4): (2, 2, 2, 2)}


def _handle(L, seed, bc_t=-1.0, **kw):
    U = inputs.gauge_field(L, 0.5, seed)
    return U, GPU(U, m0=-0.3, c_sw=1.5, mu=0.01, bc_t=bc_t, nv=8, agg=AGG[L], sap_block=AGG[L],
                  cycle_prec=F32, max_rhs=8, **kw)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 4, 10)])
@pytest.mark.parametrize("bc_t", [-1.0, 1.0])
@pytest.mark.parametrize("prec,tol", [(F32, 1e-5), (F16, 5e-3)])
def test_forward_against_oracle(L, bc_t, prec, tol):
    U, g = _handle(L, 3, bc_t)
    W1, W2 = _weights(5)
    tm.tm_nn_set_weights(g.h, nn.pack_weights(W1, W2))
    r = _fields(L, 3, 7)
    fin = g.pack(0, F32, r, 3)
    fout = g.field(0, F32, 3)
    tm.tm_nn_apply(g.h, prec, fin, fout, 3)
    got = g.unpack(0, F32, fout, r.shape, 3)
    for k in range(3):
        assert rel(got[k], nn.network(U, r[k], W1, W2, bc_t)) <= tol
    # accumulate: out += N(in)
    tm.tm_nn_apply(g.h, prec, fin, fout, 3, True)
    got2 = g.unpack(0, F32, fout, r.shape, 3)
    assert rel(got2, 2 * got) <= 1e-6


def test_wilson_weights_reproduce_dirac_operator():
    L = (4, 4, 4, 8)
    U, g = _handle(L, 11)
    W1 = np.zeros((nn.HIDDEN, 1, nn.NDIR, 4, 4), dtype=complex)
    W1[0, 0, 0] = np.eye(4)                      # hidden channel 0 = input
    W2 = np.zeros((1, nn.HIDDEN, nn.NDIR, 4, 4), dtype=complex)
    W2[0, 0] = nn.wilson_weights(-0.3)[0, 0]
    tm.tm_nn_set_weights(g.h, nn.pack_weights(W1, W2))
    assert np.array_equal(tm.tm_nn_get_weights(g.h), nn.pack_weights(W1, W2))
    psi = _fields(L, 1, 12)
    fout = g.field(0, F32)
    tm.tm_nn_apply(g.h, F32, g.pack(0, F32, psi), fout, 1)
    got = g.unpack(0, F32, fout, psi.shape)
    assert rel(got[0], Operator(U, -0.3, 0.0, 0.0).apply(psi[0])) <= 1e-6


@pytest.mark.parametrize("npairs", [1, 5, 18])
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 6, 4, 10)])
def test_loss_and_gradient_against_oracle(npairs, L):
    U, g = _handle(L, 21)
    W1, W2 = _weights(22)
    tm.tm_nn_set_weights(g.h, nn.pack_weights(W1, W2))
    R = _fields(L, npairs, 23)
    E = _fields(L, npairs, 24)
    loss, grad = tm.tm_nn_grad(g.h, g.pack(0, F32, R, npairs), g.pack(0, F32, E, npairs), npairs)
    # the oracle sees the same FP32-rounded inputs
    R32 = R.astype(np.complex64).astype(complex)
    E32 = E.astype(np.complex64).astype(complex)
    l0, G1, G2 = nn.loss_and_grad(U, R32, E32, W1, W2)
    assert abs(loss - l0) <= 1e-5 * l0
    assert rel(grad, nn.pack_weights(G1, G2)) <= 1e-4


def test_training_pairs_against_oracle_kcycle():
    L = (4, 4, 4, 4)
    U, g = _handle(L, 31, coarse_tol=0.0, coarse_maxit=6, post_smooth=2)
    tv = inputs.random_test_vectors(L, 8, 31 + inputs.TV_SEED_OFFSET)
    tm.tm_setup_from_vectors(g.h, tv)
    p = g.p
    prm = AMGParams(m0=-0.3, c_sw=1.5, mu=0.01, delta=p.delta, nv=8, agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2),
                    mr_iters=p.mr_iters, pre_smooth=p.pre_smooth, post_smooth=p.post_smooth,
                    coarse_tol=0.0, coarse_restart=p.coarse_restart, coarse_maxit=6)
    tl = TwoLevel(U, prm)
    tl.build_coarse(tv)
    e0 = inputs.gaussian_spinor(L, 32, nrhs=3)
    fr, fe = g.field(0, F32, 3), g.field(0, F32, 3)
    tm.tm_nn_pairs(g.h, e0, fr, fe, 3)
    got_r = g.unpack(0, F32, fr, e0.shape, 3)
    got_e = g.unpack(0, F32, fe, e0.shape, 3)
    for k in range(3):
        e = e0[k] - tl.kcycle(tl.op.apply(e0[k]))
        assert rel(got_e[k], e) <= 1e-4
        assert rel(got_r[k], tl.op.apply(e)) <= 1e-4


def _trained(L, seed, npairs=24, epochs=40):
    U, g = _handle(L, seed, setup_iters=2)
    tv = inputs.random_test_vectors(L, 8, seed + inputs.TV_SEED_OFFSET)
    tm.tm_setup(g.h, tv)
    W1, W2 = _weights(seed + 1, 0.02)
    tm.tm_nn_set_weights(g.h, nn.pack_weights(W1, W2))
    e0 = inputs.gaussian_spinor(L, seed + 2, nrhs=npairs)
    fr, fe = g.field(0, F32, npairs), g.field(0, F32, npairs)
    tm.tm_nn_pairs(g.h, e0, fr, fe, npairs)
    losses = tm.tm_nn_train(g.h, fr, fe, npairs, epochs, 8, 3e-3)
    return U, g, tv, losses


def test_adam_training_lowers_the_loss():
    U, g, tv, losses = _trained((8, 4, 4, 4), 41)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.9 * losses[0], losses


@pytest.mark.parametrize("mode,prec", [(1, F32), (1, F16), (2, F32)])
def test_solve_with_stage_after_kcycle(mode, prec):
    L = (8, 4, 4, 4)
    U, g, tv, losses = _trained(L, 51, npairs=16, epochs=20)
    w = tm.tm_nn_get_weights(g.h)
    U2 = U
    h2 = GPU(U2, m0=-0.3, c_sw=1.5, mu=0.01, nv=8, agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), cycle_prec=F32,
             max_rhs=2, setup_iters=2, nn_mode=mode, nn_prec=prec)
    tm.tm_setup(h2.h, tv)
    tm.tm_nn_set_weights(h2.h, w)
    b = inputs.gaussian_spinor(L, 52, nrhs=2)
    x = np.zeros_like(b)
    st, info = tm.tm_solve(h2.h, b, x, 2, 1e-10)
    assert st == tm.TM_OK and info.converged and info.true_relres <= 1e-10
    op = Operator(U, -0.3, 1.5, 0.01)
    for k in range(2):
        assert np.linalg.norm(b[k] - op.apply(x[k])) / np.linalg.norm(b[k]) <= 1e-10


def test_adam_steps_match_numpy_restatement():
    """tm_nn_train's update, restated in numpy: Adam (beta1 0.9, beta2 0.999,
    eps 1e-8, bias-corrected) on the real and imaginary parts of every weight
    with the steepest-descent direction 2 dL/d conj(W) of each minibatch, in
    order.  The restatement is fed the library's own minibatch gradients
    (tm_nn_grad at the restated weights; those gradients are checked against
    the oracle above), so the comparison isolates the update rule."""
    L = (4, 4, 4, 4)
    U, g = _handle(L, 61)
    _, g_ref = _handle(L, 61)
    W1, W2 = _weights(62, 0.05)
    w = nn.pack_weights(W1, W2)
    npairs, batch, epochs, lr = 8, 3, 2, 2e-3
    R = _fields(L, npairs, 63)
    E = _fields(L, npairs, 64)
    fr, fe = g.pack(0, F32, R, npairs), g.pack(0, F32, E, npairs)
    tm.tm_nn_set_weights(g.h, w)
    tm.tm_nn_train(g.h, fr, fe, npairs, epochs, batch, lr)
    got = tm.tm_nn_get_weights(g.h)
    fb = tm.tm_field_bytes(g.h, 0, F32, 1)
    m = np.zeros(2 * w.size)
    v = np.zeros(2 * w.size)
    t = 0
    b1, b2, eps = 0.9, 0.999, 1e-8
    for _ in range(epochs):
        for p0 in range(0, npairs, batch):
            nb = min(batch, npairs - p0)
            tm.tm_nn_set_weights(g_ref.h, w)
            _, G = tm.tm_nn_grad(g_ref.h, fr[p0 * fb:(p0 + nb) * fb], fe[p0 * fb:(p0 + nb) * fb], nb)
            gr = np.empty(2 * w.size)
            gr[0::2], gr[1::2] = 2 * G.real, 2 * G.imag
            t += 1
            m = b1 * m + (1 - b1) * gr
            v = b2 * v + (1 - b2) * gr * gr
            upd = lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
            w = w - (upd[0::2] + 1j * upd[1::2])
    assert t == 6
    assert rel(got, w) <= 1e-12
    # and the update moved the weights by about lr per component and step
    assert rel(got, nn.pack_weights(W1, W2)) > 1e-3
