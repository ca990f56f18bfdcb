"""The learned warm start on the time march it was built for: 2D channel 128x32, dG(1),
tau = 0.005, 400 slabs; the network is trained on the GPU on slabs 1-200 and every slab
of 201-400 is solved from three initial guesses to the same absolute tolerances
(Newton 1e-8, GMRES 1e-9, as in Sec. 4):

* fallback: the previous slab's end value at every Radau node (no learned part);
* linear:   linear extrapolation from the end values of the last two slabs;
* network:  linear extrapolation plus the trained network's correction.
"""
import numpy as np
import pytest

import stg_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def march():
    from paper_2210_02690_gb300.march import March
    cfg = si.MARCH
    m = March(cfg["spec"], cfg["k"], cfg["nu"], cfg["tau"], si.march_initial_velocity(cfg["spec"], pert=cfg["pert"]),
              si.march_inflow(cfg["spec"], cfg["k"]), vcycle_prec="f32", factor_prec="f32")
    m.run(cfg["slabs"])
    yield m
    m.close()


def test_march_converges_every_slab(march):
    assert len(march.X) == si.MARCH["slabs"] + 1
    assert all(r["res"] <= 1e-8 for r in march.stats)


def test_network_warm_start_beats_the_fallback(march):
    from paper_2210_02690_gb300.march import summary
    cfg = si.MARCH
    n_train = cfg["train_slabs"]
    net, sv, losses, _ = march.train(cfg["channels"], si.cnn_init(cfg["channels"]), list(range(2, n_train)))
    assert np.median(losses[-20:]) < 0.1 * losses[0]
    ev = march.evaluate(list(range(n_train, cfg["slabs"])), net, sv)
    s = {name: summary(rows) for name, rows in ev.items()}
    for name, v in s.items():
        assert v["all_converged"] and v["max_final_over_tol"] <= 1.0, name
    fb, lin, nw = s["fallback"], s["linear"], s["network"]
    # what the trained network gains over the method without it
    assert nw["newton_steps"] <= fb["newton_steps"]
    assert nw["gmres_iters"] < 0.75 * fb["gmres_iters"]
    assert nw["mean_r0"] < 0.1 * fb["mean_r0"]
    # and over its own linear-extrapolation part
    assert nw["mean_r0"] < 0.8 * lin["mean_r0"]
    assert nw["gmres_iters"] <= lin["gmres_iters"]
    net.close()


def test_guesses_at_tight_tolerances_and_plain_f64(march):
    """At Newton 1e-10 / GMRES 1e-11 absolute the initial guess decides how many GMRES iterations a
    slab needs: the network's guess needs no more than the linear extrapolation and fewer than the
    fallback; the warm-started FP32 form needs no more GMRES iterations than the plain FP64 form
    solved from the fallback guess at the paper's tolerances."""
    from paper_2210_02690_gb300.march import summary
    cfg = si.MARCH
    n_train = cfg["train_slabs"]
    net, sv, _, _ = march.train(cfg["channels"], si.cnn_init(cfg["channels"]), list(range(2, n_train)))
    slabs = list(range(n_train, n_train + 60))
    tight = march.companion_solver(vcycle_prec="f32", factor_prec="f32", gmres_atol=1e-11)
    ev = march.evaluate(slabs, net, sv, solver=tight, atol=1e-10)
    tight.close()
    s = {name: summary(rows) for name, rows in ev.items()}
    for name, v in s.items():
        assert v["all_converged"] and v["max_final_over_tol"] <= 1.0, name
    assert s["network"]["gmres_iters"] <= s["linear"]["gmres_iters"]
    assert s["network"]["gmres_iters"] < s["fallback"]["gmres_iters"]
    f64 = march.companion_solver(vcycle_prec="f64", factor_prec="f64")
    ev64 = march.evaluate(slabs, net, sv, solver=f64, names=("fallback",))
    f64.close()
    warm = march.evaluate(slabs, net, sv, names=("network",))
    assert summary(warm["network"])["gmres_iters"] <= summary(ev64["fallback"])["gmres_iters"]
    net.close()
