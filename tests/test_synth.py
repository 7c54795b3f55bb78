"""The synthetic workload generators (no method arithmetic): the SDF field of the mesh-extraction
workload, its torch twin used for fitting, and the folded SIREN initialisation."""
import numpy as np
import pytest

from synth import fields, inr


def test_sdf_field_signs_and_torch_twin():
    f = fields.torus_and_spheres()
    inside = np.array([[0.5, 0.0, 0.0], [-0.25, 0.43, 0.1], [0.0, 0.0, 0.45], [0.0, -0.5, 0.0]])
    outside = np.array([[0.0, 0.0, 0.0], [0.95, 0.95, 0.95], [0.0, 0.0, -0.9]])
    assert np.all(f(inside) < 0) and np.all(f(outside) > 0)
    # on the torus's ring away from the spheres the value is minus the minor radius
    assert abs(f(np.array([[0.0, -0.5, 0.0]]))[0] + 0.18) < 1e-12
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).uniform(-1, 1, size=(500, 3))
    np.testing.assert_allclose(f.torch_eval(torch.tensor(x)).numpy(), f(x), rtol=1e-12, atol=1e-12)


def test_siren_initialisation_folds_omega0():
    layers = inr.siren_init([3, 64, 64, 1], 3, omega0=30.0)
    (W0, b0), (W1, b1), (W2, b2) = layers
    assert np.abs(W0).max() <= 30.0 / 3 + 1e-5                       # omega0 x U(+-1/fan_in)
    assert np.abs(W1).max() <= np.sqrt(6.0 / 64) + 1e-5             # omega0 x U(+-sqrt(6/fan_in)/omega0)
    assert np.abs(W2).max() <= np.sqrt(6.0 / 64) / 30.0 + 1e-6       # output layer not folded
    assert np.abs(b0).max() <= 30.0 / np.sqrt(3) + 1e-4 and np.abs(b2).max() <= 1 / 8 + 1e-6
    assert inr.random_inr([3, 64, 64, 1], 3, act="sine")[0][0].shape == (64, 3)
