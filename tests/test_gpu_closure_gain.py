"""What the learned closure gains over plain Smagorinsky (the method without it).

A fine channel (256 x 128 x 128, Re_tau ~ 180, bulk velocity 0.1) is spun up with the
Smagorinsky closure; 20 box-filtered sample sets train the network with the library's own
kernels.  Then:
  * a priori: on held-out (later) snapshots the network's eddy-viscosity error must be at
    most half of Smagorinsky's (the zero output layer);
  * a posteriori: coarse 128 x 64 x 64 runs from the filtered fine state, Smagorinsky vs
    the learned closure (Smagorinsky as its lower bound), against the filtered fine run over
    20000 coarse steps: the learned closure must stay stable and its combined profile error
    (mean u_x plus RMS velocity, relative) must be below Smagorinsky's.
"""
import pytest

pytestmark = pytest.mark.gpu


def test_learned_closure_gains_over_smagorinsky():
    import torch

    from paper_2305_09910_gb300 import build, closure

    assert torch.cuda.is_available()
    build.build()
    rep = closure.experiment(256, 128, 128, re_tau=180.0, u_bulk=0.1, spin=60000, nsnap=20,
                             every=500, epochs=6, coarse_steps=20000, cs_min=0.1)
    assert rep["apriori_gain"] >= 0.5, rep["apriori_gain"]
    ap = rep["aposteriori"]
    assert "unstable" not in ap["mlp"] and "unstable" not in ap["smag"], ap
    err = {k: ap[k]["mean_err"] + ap[k]["rms_err"] for k in ("smag", "mlp")}
    print("closure experiment:", {k: v for k, v in rep.items() if k != "params"})
    assert err["mlp"] < err["smag"], err
