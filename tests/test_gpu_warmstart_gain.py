"""What the learned warm start gains, measured on held-out drops.

The network (trained on the GPU by the library's kernels on solver-made
steady states) starts a run closer to the solver's steady density than the
tanh profile does, and at least 80% of the held-out runs end in the tanh
start's steady state (the solver has the last word; a heuristic start can send
a drop elsewhere, which is counted and printed).  Steps to the steady-state
check are measured and printed: they are about the same from either start,
so no speed-up is asserted.
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
    ok = [k for k in range(len(held)) if st_tanh[k] == 0 and st_warm[k] == 0]
    assert len(ok) >= 10
    e_tanh, e_warm, same = [], [], []
    with lb.Batch([held[k] for k in ok], W.A_VDW, W.B_VDW, scheme=lb.FORCING) as bt:
        bt.init_drops(2.0)
        for j, k in enumerate(ok):
            start = bt.fields(j)[0]
            steady = f_tanh[k][0]
            rho_w, _ = W.predict_start(ws, start, held[k], use_u=False)
            e_tanh.append(np.sqrt(np.mean((start - steady) ** 2)))
            e_warm.append(np.sqrt(np.mean((rho_w - steady) ** 2)))
            same.append(np.abs(f_warm[k][0] - steady).max() < 1e-4)
    # the network is a heuristic start: most runs must end in the tanh start's steady state
    assert sum(same) >= 0.8 * len(ok)
    sel = [j for j in range(len(ok)) if same[j]]
    gain = np.mean([e_warm[j] for j in sel]) / np.mean([e_tanh[j] for j in sel])
    ratio = np.mean([s_warm[ok[j]] for j in sel]) / np.mean([s_tanh[ok[j]] for j in sel])
    print(f"{sum(same)}/{len(ok)} reach the same steady state; initial rms density error warm/tanh = "
          f"{gain:.3f}; steps to steady warm/tanh = {ratio:.3f}")
    assert gain < 0.8
    ws.close()
