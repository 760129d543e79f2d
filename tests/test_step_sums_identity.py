"""The identity behind the fused step sums (lbm_step_reduce), checked with the oracle's
propagation (Eq. 16 with halfway bounce-back) on the CPU.

Streaming maps post-collision populations one to one onto the new state; a population
whose link leaves through a wall comes back into its own cell reversed.  So the sum of
phi over the new state equals the sum of all post-collision f, and the new lattice
momentum equals sum c'_i g_i^+ with c'_i = -c_i for the populations that bounce.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O


def _post(q, shape, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(q,) + shape)


@pytest.mark.parametrize("walls", [False, True])
def test_mass_is_the_sum_of_post_collision_values(walls):
    post = _post(7, (6, 5, 4), 1)
    new = O.stream(post, O.D3Q7_C, O.opposite(O.D3Q7_C), walls)
    assert np.isclose(new.sum(), post.sum(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("nz", [1, 2, 7])
def test_momentum_with_bounced_populations_negated(nz):
    post = _post(15, (nz, 5, 4), 2)
    C = O.D3Q15_C.astype(np.float64)
    new = O.stream(post, O.D3Q15_C, O.opposite(O.D3Q15_C), True)
    after = np.einsum("ia,i...->a...", C, new).reshape(3, -1).sum(axis=1)
    z = np.arange(nz)[None, :, None, None]
    cz = C[:, 2][:, None, None, None]
    bounces = ((cz > 0) & (z == nz - 1)) | ((cz < 0) & (z == 0))
    sign = np.where(bounces, -1.0, 1.0)
    fused = np.einsum("ia,i...->a...", C, sign * post).reshape(3, -1).sum(axis=1)
    np.testing.assert_allclose(fused, after, rtol=0, atol=1e-11)
    # without the correction the momentum is wrong by twice the walls' share
    plain = np.einsum("ia,i...->a...", C, post).reshape(3, -1).sum(axis=1)
    assert abs(plain[2] - after[2]) > 1.0
