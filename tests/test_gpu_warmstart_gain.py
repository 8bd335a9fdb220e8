"""What the learned warm start gains, measured on held-out drops.

The network (trained on the GPU by the library's kernels on solver-made
steady states) starts a run closer to the solver's steady density than the
tanh profile does, and every held-out run reaches the tanh start's steady
state from it: the same bulk densities, equimolar radius and spurious
velocity, with the drop left where it started (the solver has the last word;
a start that sets the drop moving excites the translation mode of the
periodic lattice, which steady.fast detects and hands back to the tanh start).
Steps to the steady-state check are measured and bounded: the network's start
costs at most 5% more steps than the tanh start (measured 1.02 over two
trainings) - it is not a speed-up.
"""
import numpy as np
import pytest

from paper_0710_5470_gb300 import inputs
from tests.helpers import library

pytestmark = pytest.mark.gpu


def test_warm_start_is_closer_to_steady_state():
    lb = library()
    from paper_0710_5470_gb300 import warmstart as W
    sweep = inputs.sweep_instances(seed=11, count=272, side=(48, 48), T=(0.53, 0.56), kappa=(0.005, 0.015),
                                   tau=(0.7, 1.2), rfrac=(0.2, 0.35))
    inst = W.instances_from_sweep(sweep)
    train_set, held = inst[:256], inst[256:]
    x, t, keep, _ = W.steady_dataset(train_set, tol=1e-8, every=50, max_steps=40000)
    assert len(keep) >= 200
    ws, hist = W.train(x, t, epochs=300, batch=16, lr=1e-3)
    assert hist[-1] < 0.7 * hist[0]
    s_tanh, st_tanh, f_tanh = W.steps_to_steady(held, None, tol=1e-8, every=50, max_steps=40000)
    s_warm, st_warm, f_warm = W.steps_to_steady(held, ws, tol=1e-8, every=50, max_steps=40000, use_u=False)
    ok = [k for k in range(len(held)) if st_tanh[k] == 0]
    assert len(ok) >= 10
    e_tanh, e_warm = [], []
    with lb.Batch([held[k] for k in ok], W.A_VDW, W.B_VDW, scheme=lb.FORCING) as bt:
        bt.init_drops(2.0)
        for j, k in enumerate(ok):
            start = bt.fields(j)[0]
            steady = f_tanh[k][0]
            rho_w, _ = W.predict_start(ws, start, held[k], use_u=False)
            e_tanh.append(np.sqrt(np.mean((start - steady) ** 2)))
            e_warm.append(np.sqrt(np.mean((rho_w - steady) ** 2)))
    ws.close()
    for k in ok:
        assert st_warm[k] == 0, k                       # converges from the network's start too
    # where both runs end up: each final state settled in float64 to 1e-11 (uncounted)
    set_t = W.settle([held[k] for k in ok], [f_tanh[k] for k in ok])
    set_w = W.settle([held[k] for k in ok], [f_warm[k] for k in ok])
    cmp = []
    for j, k in enumerate(ok):
        rl, rg = lb.coexistence(W.A_VDW, W.B_VDW, held[k]["T"])
        cmp.append(W.same_steady_state(set_t[j], set_w[j], rl, rg))
    gain = np.mean(e_warm) / np.mean(e_tanh)
    ratio = sum(s_warm[k] for k in ok) / sum(s_tanh[k] for k in ok)
    print(f"{sum(c['same'] for c in cmp)}/{len(ok)} reach the same steady state (largest drift "
          f"{max(c['shift'] for c in cmp):.2e} sites, largest pointwise difference "
          f"{max(c['pointwise'] for c in cmp):.2e}); initial rms density error warm/tanh = {gain:.3f}; "
          f"steps to steady warm/tanh = {ratio:.3f}")
    assert all(c["same"] for c in cmp)
    assert all(c["shift"] < 0.5 for c in cmp)
    assert gain < 0.8
    assert ratio <= 1.05
