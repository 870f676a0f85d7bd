"""The closed-loop plant (gato_plant_rk4 / gato_plant_ee, host FP64) against
the oracle's dynamics: one RK4 step of the plant equals RK4 composed from the
oracle's forward dynamics, with and without an end-effector force, and the
plant's end-effector position equals the oracle's forward kinematics.  The
plant is host code: these run without a GPU.
"""
import numpy as np
import pytest

from paper_2510_07625_gb300 import inputs as I

MODELS = [I.arm7(), I.arm6(),
          I.chain([0, 2], [0.3, 0.2], [1.2, 0.8], inertia_diag=[0.01, 0.02, 0.03, 0.004, 0.005, 0.006],
                  com=[0.01, -0.02, 0.12, 0.03, 0.0, 0.05], name="2xz_offset_com")]


@pytest.fixture(scope="module")
def G():
    from paper_2510_07625_gb300 import build, gato

    build.build_library()
    gato.load()
    return gato


def f32(model):
    """The model with its parameters rounded to float32, as gato_model_desc holds them."""
    r = lambda t: tuple(float(np.float32(v)) for v in t)
    return I.ArmModel(model.dof, model.axis, r(model.link_len), r(model.mass), r(model.com),
                      r(model.inertia), float(np.float32(model.gravity)), model.name)


def _rk4_oracle(oracle, model, x, u, h, f):
    n = model.dof

    def fn(y):
        return np.concatenate([y[n:], oracle.forward_dynamics(model, y[:n], y[n:], u, f_ext=f)])
    k1 = fn(x)
    k2 = fn(x + 0.5 * h * k1)
    k3 = fn(x + 0.5 * h * k2)
    k4 = fn(x + h * k3)
    return x + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)


@pytest.mark.parametrize("model", MODELS, ids=lambda m: m.name)
@pytest.mark.parametrize("force", [None, (15.0, -20.0, -50.0)])
def test_plant_rk4_matches_oracle(G, oracle, model, force):
    plant = G.Plant(model)
    rng = np.random.default_rng(31)
    n = model.dof
    for _ in range(3):
        x = np.concatenate([rng.uniform(-1.5, 1.5, n), rng.uniform(-2, 2, n)])
        u = rng.uniform(-20, 20, n)
        h = 1e-3
        got = plant.rk4(x, u, h, 1, f_ext=force)
        want = _rk4_oracle(oracle, f32(model), x, u, h, None if force is None else np.array(force))
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)
        # several steps = the steps one at a time
        many = plant.rk4(x, u, h, 5, f_ext=force)
        y = x
        for _ in range(5):
            y = plant.rk4(y, u, h, 1, f_ext=force)
        np.testing.assert_array_equal(many, y)


@pytest.mark.parametrize("model", MODELS, ids=lambda m: m.name)
def test_plant_ee_matches_oracle_fk(G, oracle, model):
    plant = G.Plant(model)
    rng = np.random.default_rng(32)
    for _ in range(5):
        q = rng.uniform(-2, 2, model.dof)
        np.testing.assert_allclose(plant.ee(q), oracle.fk(f32(model), q), rtol=0, atol=1e-13)


def test_plant_rejects_bad_arguments(G):
    plant = G.Plant(I.arm7())
    x = np.zeros(14)
    with pytest.raises(G.GatoError):
        plant.rk4(x, np.zeros(7), 0.0, 1)
    with pytest.raises(G.GatoError):
        plant.rk4(x, np.zeros(7), 1e-3, -1)
    np.testing.assert_array_equal(plant.rk4(x + 0.1, np.zeros(7), 1e-3, 0), x + 0.1)
