"""Pins of the BF16-operand variant of the network oracle: the rounding itself, and the variant
reducing to the FP64 network when the rounding is the identity."""
import numpy as np

from oracle import mlp as omlp


def test_bf16_rounding_values():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even neighbour (1)
    assert omlp.bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: even neighbour 1 + 2^-6
    assert omlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert omlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert omlp.bf16(-3.0) == -3.0 and omlp.bf16(0.0) == 0.0
    x = np.random.default_rng(0).normal(size=1000)
    r = omlp.bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))          # within half a BF16 ulp
    assert np.array_equal(omlp.bf16(r), r)                         # idempotent


def test_identity_rounding_reduces_to_the_fp64_network():
    rng = np.random.default_rng(3)
    theta = rng.normal(0, 0.1, omlp.n_params())
    X = rng.uniform(-1, 1, (40, 16))
    Y = rng.normal(0, 0.5, (40, 3))
    ident = lambda a: np.asarray(a, dtype=np.float64)
    p1, _ = omlp.forward(theta, X)
    p2, _ = omlp.forward_bf16(theta, X, ident)
    np.testing.assert_allclose(p2, p1, rtol=1e-13, atol=1e-15)
    l1, g1 = omlp.loss_and_grad(theta, X, Y)
    l2, g2, s2 = omlp.loss_and_grad_bf16(theta, X, Y, ident)
    assert abs(l1 - l2) <= 1e-14 * l1
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-16)
    assert np.all(s2 >= np.abs(g2) - 1e-15)
