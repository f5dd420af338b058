"""Batched serving and CUDA-graph replay: every reconstruction of a batched call
equals its own standalone epoch (and the FP64 oracle), and graph-replayed
epochs equal eager ones over several calls in a row."""
import math

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2510_20929_gb300 import synth
from tests.parity_util import TOL_EPOCH, c64, err, f32pos, problem, to_dev

pytestmark = pytest.mark.gpu


def _gpu_inputs(shapes):
    """Seeded small problems of uneven size, on the device."""
    import torch
    out = []
    for i, (N, M, H, W, J, step, B) in enumerate(shapes):
        p = problem(N=N, M=M, H=H, W=W, J=J, step=step, seed=40 + i)
        O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
        order = np.random.default_rng(i).permutation(J).astype(np.int32)
        out.append(dict(np=(O, P, pos, I_m, order, B),
                        dev=(to_dev(O, torch.complex64), to_dev(P, torch.complex64), to_dev(pos, torch.float32),
                             to_dev(I_m, torch.float32), to_dev(order, torch.int32))))
    return out


SHAPES = [(32, 2, 72, 76, 16, 6.0, 6), (64, 1, 150, 160, 20, 12.0, 8), (16, 3, 41, 37, 9, 3.0, 9),
          (64, 3, 160, 150, 25, 12.0, 10), (128, 2, 300, 310, 12, 24.0, 5), (192, 1, 256, 266, 6, 20.0, 4),
          (256, 2, 320, 330, 5, 20.0, 3)]


@pytest.mark.parametrize("graph", [False, True])
def test_batched_equals_standalone_and_oracle(graph):
    import torch
    from paper_2510_20929_gb300 import api
    items = _gpu_inputs(SHAPES)
    ref = []
    for it in items:
        O, P, pos, meas, order = (t.clone() for t in it["dev"])
        B = it["np"][5]
        loss, _ = api.lsqml_epoch(O, P, pos, meas, order, batch=B, delta_o=0.1, delta_p=0.1, eps=1e-6)
        ref.append((O, P, loss.item()))
    recons, opts = [], []
    for it in items:
        O, P, pos, meas, order = (t.clone() for t in it["dev"])
        recons.append((O, P, pos, meas, order))
        opts.append(api.make_opts(batch=it["np"][5], delta_o=0.1, delta_p=0.1, eps=1e-6, graph=graph))
    losses = api.lsqml_epoch_batched(recons, opts)
    for i, ((O, P, *_), (Or, Pr, Lr)) in enumerate(zip(recons, ref)):
        e = (err(O.cpu().numpy(), Or.cpu().numpy()), err(P.cpu().numpy(), Pr.cpu().numpy(), axis=0),
             abs(losses[i].item() - Lr) / abs(Lr))
        print(f"recon {i}: {e}")
        assert max(e) < TOL_EPOCH
    # one of them against the oracle
    O, P, pos, I_m, order, B = items[0]["np"]
    O_ref, P_ref, _, _ = orc.lsqml_epoch(O, P, pos, I_m, order,
                                         orc.LsqmlOptions(batch=B, delta_o=0.1, delta_p=0.1, eps=1e-6))
    assert err(recons[0][0].cpu().numpy(), O_ref) < TOL_EPOCH and err(recons[0][1].cpu().numpy(), P_ref, axis=0) < TOL_EPOCH


def test_graph_replay_equals_eager_over_consecutive_epochs():
    import torch
    from paper_2510_20929_gb300 import api
    it = _gpu_inputs([SHAPES[3]])[0]
    O0, P0, pos, meas, order = it["dev"]
    Oe, Pe, Og, Pg = O0.clone(), P0.clone(), O0.clone(), P0.clone()
    eager = api.make_opts(batch=10, delta_o=0.1, delta_p=0.1, eps=1e-6)
    graphed = api.make_opts(batch=10, delta_o=0.1, delta_p=0.1, eps=1e-6, graph=True)
    for epoch in range(4):
        le, _ = api.lsqml_epoch(Oe, Pe, pos, meas, order, eager)
        lg, _ = api.lsqml_epoch(Og, Pg, pos, meas, order, graphed)
        e = (err(Og.cpu().numpy(), Oe.cpu().numpy()), err(Pg.cpu().numpy(), Pe.cpu().numpy(), axis=0),
             abs(lg.item() - le.item()) / abs(le.item()))
        print(f"epoch {epoch}: {e}")
        assert max(e) < TOL_EPOCH


def test_uneven_workload_generator_stays_in_bounds():
    ws = synth.workload_uneven(16, J_range=(500, 20000))
    for w in ws:
        s = w["pos"] - w["N"] / 2.0
        assert s.min() >= 0 and s.max() < w["H"] - w["N"]


def test_autotuned_epoch_matches_default_and_records_its_choice():
    from paper_2510_20929_gb300 import api
    it = _gpu_inputs([SHAPES[1]])[0]
    O0, P0, pos, meas, order = it["dev"]
    Od, Pd, Ot, Pt = O0.clone(), P0.clone(), O0.clone(), P0.clone()
    ld, _ = api.lsqml_epoch(Od, Pd, pos, meas, order, api.make_opts(batch=8, delta_o=0.1, delta_p=0.1, eps=1e-6))
    lt, _ = api.lsqml_epoch(Ot, Pt, pos, meas, order,
                            api.make_opts(batch=8, delta_o=0.1, delta_p=0.1, eps=1e-6, autotune=True))
    e = (err(Ot.cpu().numpy(), Od.cpu().numpy()), err(Pt.cpu().numpy(), Pd.cpu().numpy(), axis=0),
         abs(lt.item() - ld.item()) / abs(ld.item()))
    t = api.tuning(api.dims_of(O0, P0, pos), 8)
    print("autotune:", e, t)
    assert max(e) < TOL_EPOCH
    assert t is not None and t["pass1"] in (0, 1) and t["pass2"] in (0, 1, 2, 3) and t["probe_reduce"] in (0, 1, 2, 3)
    assert min(t["pass1_ms"][:2]) > 0 and min(t["pass2_ms"][:4]) > 0 and min(t["probe_reduce_ms"][:4]) > 0
