"""The allocation-free epoch entry point (ptycho_lsqml_epoch_static).

Callers that cannot allocate device memory (applications that hand the whole
device memory budget to their own allocator up front, or real-time pipelines
that must not call cudaMalloc because it can synchronise the device) use this
entry point: it runs the same LSQML epoch as ptycho_lsqml_epoch with its
scratch in a fixed device array inside the library. These tests call it
through the C ABI and compare it with the workspace entry point. The file is
named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from tests.parity_util import TOL_EPOCH, c64, err, f32pos, problem, to_dev



def test_static_entry_rejects_problems_beyond_its_capacity():
    # host-side check, before any CUDA call: the spiral workload at batch 256
    # needs far more than PTYCHO_STATIC_WS_BYTES of scratch
    from paper_2510_20929_gb300 import api
    L = api.lib()
    d = api.Dims(1024, 1024, 128, 5, 4096)
    opts = api.make_opts(batch=256)
    fake = ctypes.c_void_p(0x1000)     # never dereferenced
    assert L.ptycho_workspace_bytes(ctypes.byref(d), 256) > 64 * 1024 * 1024
    st = L.ptycho_lsqml_epoch_static(ctypes.byref(d), fake, fake, fake, fake, None, ctypes.byref(opts),
                                     None, None, None)
    assert st == 8 and "static" in api.status_string(st)


def _inputs(N, M, H, W, J, step, seed):
    import torch
    p = problem(N=N, M=M, H=H, W=W, J=J, step=step, seed=seed)
    O, P, pos, I_m = c64(p["O"]), c64(p["P"]), f32pos(p["pos"]), np.float32(p["I_m"]).astype(np.float64)
    order = np.random.default_rng(seed).permutation(J).astype(np.int32)
    return (to_dev(O, torch.complex64), to_dev(P, torch.complex64), to_dev(pos, torch.float32),
            to_dev(I_m, torch.float32), to_dev(order, torch.int32))


@pytest.mark.gpu
def test_static_scratch_epoch_matches_workspace_epoch_on_consecutive_calls():
    import torch
    from paper_2510_20929_gb300 import api
    L = api.lib()
    cases = [((32, 2, 72, 76, 16, 6.0, 7), 6), ((32, 2, 72, 76, 16, 6.0, 7), 6), ((64, 3, 150, 160, 20, 12.0, 9), 8)]
    for (args, batch) in cases:
        O0, P0, pos, meas, order = _inputs(*args)
        opts = api.make_opts(batch=batch, delta_o=0.1, delta_p=0.1, lam=1e-6, eps=1e-6)
        O_ref, P_ref = O0.clone(), P0.clone()
        loss_ref, alpha_ref = api.lsqml_epoch(O_ref, P_ref, pos, meas, order, opts, want_alpha=True)
        O, P = O0.clone(), P0.clone()
        loss = torch.zeros((), dtype=torch.float64, device=O.device)
        alpha = torch.zeros((pos.shape[0], 2), dtype=torch.float64, device=O.device)
        d = api.dims_of(O, P, pos)
        st = L.ptycho_lsqml_epoch_static(ctypes.byref(d), ctypes.c_void_p(O.data_ptr()),
                                         ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(pos.data_ptr()),
                                         ctypes.c_void_p(meas.data_ptr()), ctypes.c_void_p(order.data_ptr()),
                                         ctypes.byref(opts), ctypes.c_void_p(loss.data_ptr()),
                                         ctypes.c_void_p(alpha.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == 0, api.status_string(st)
        e = (err(O.cpu().numpy(), O_ref.cpu().numpy()), err(P.cpu().numpy(), P_ref.cpu().numpy(), axis=0),
             err(alpha.cpu().numpy(), alpha_ref.cpu().numpy(), axis=1),
             abs(loss.item() - loss_ref.item()) / abs(loss_ref.item()))
        print("static vs workspace:", e)
        assert max(e) < TOL_EPOCH
