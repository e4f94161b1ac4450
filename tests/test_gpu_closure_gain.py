"""What the learned closure gains over plain Smagorinsky (the method without it), over seeds.

For each of three seeds (network initialisation, minibatch order and the perturbations of
the initial flow), a fine channel (256 x 128 x 128, Re_tau ~ 180, bulk velocity 0.1, initial
sinusoid amplitude 0.5 u_b so that it becomes turbulent within the spin-up) is spun up with
the Smagorinsky closure; 20 box-filtered sample sets train the network with the library's
own kernels.  Then:
  * a priori: on held-out (later) snapshots the network's eddy-viscosity error is at most
    half of Smagorinsky's (the zero output layer), for every seed;
  * a posteriori: coarse 128 x 64 x 64 runs from the filtered fine state, Smagorinsky vs the
    learned closure (Smagorinsky as its lower bound), against the filtered fine run over
    20000 coarse steps: both stay stable.  The learned closure does NOT improve the coarse
    profiles: its combined profile error (mean u_x plus RMS velocity, relative) was higher
    than Smagorinsky's on every seed, 0.335 +- 0.022 against 0.294 +- 0.021 over the three
    seeds (+14 %).  That comparison is reported here, not claimed as a gain; the test only
    guards it from growing, holding the learned closure's mean error within 25 % of
    Smagorinsky's.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_closure_gain_over_seeds():
    import torch

    from paper_2305_09910_gb300 import build, closure, inputs

    assert torch.cuda.is_available()
    build.build()
    reps = []
    for seed in (0, 1, 2):
        rep = closure.experiment(256, 128, 128, re_tau=180.0, u_bulk=0.1, spin=60000, nsnap=20, every=500,
                                 epochs=6, coarse_steps=20000, cs_min=0.1, seed=seed, amp=0.5,
                                 flow_seed=inputs.DEFAULT_SEED + seed)
        rep.pop("params")
        reps.append(rep)
        print(f"seed {seed}:", {k: rep[k] for k in ("apriori_gain", "aposteriori", "fine_rms_max_after_spin")})
    utau = inputs.channel_parameters(128, u_bulk=0.1)["u_tau"]
    err = {}
    for rep in reps:
        assert rep["fine_rms_max_after_spin"][1] >= 0.5 * utau  # the fine run is turbulent
        assert rep["apriori_gain"] >= 0.5, rep["apriori_gain"]
        ap = rep["aposteriori"]
        assert "unstable" not in ap["mlp"] and "unstable" not in ap["smag"], ap
        for k in ("smag", "mlp"):
            err.setdefault(k, []).append(ap[k]["mean_err"] + ap[k]["rms_err"])
    e_s, e_m = np.array(err["smag"]), np.array(err["mlp"])
    print(f"combined profile error over seeds: Smagorinsky {e_s.mean():.4f} +- {e_s.std():.4f}, "
          f"learned {e_m.mean():.4f} +- {e_m.std():.4f}; a-priori gains "
          f"{[round(r['apriori_gain'], 3) for r in reps]}")
    assert e_m.mean() <= 1.25 * e_s.mean(), (e_m, e_s)
