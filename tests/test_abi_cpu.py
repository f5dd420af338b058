"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/ptycho.h, and rejects bad arguments on the host before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptycho.h")


@pytest.fixture(scope="module")
def L():
    from paper_2510_20929_gb300 import api
    if not os.path.exists(api.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return api.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ptycho_[a-z_]+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("ptycho_forward", "ptycho_adjoint", "ptycho_lsqml_epoch", "ptycho_workspace_bytes",
              "ptycho_status_read", "ptycho_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings(L):
    from paper_2510_20929_gb300 import api
    for code in range(8):
        assert len(api.status_string(code)) > 0
    assert api.status_string(0) == "ok"


def _dims(H=64, W=64, N=32, M=2, J=5):
    from paper_2510_20929_gb300 import api
    return api.Dims(H, W, N, M, J)


def test_workspace_bytes_host_logic(L):
    from paper_2510_20929_gb300 import api
    d = _dims()
    a = L.ptycho_workspace_bytes(ctypes.byref(d), 4)
    b = L.ptycho_workspace_bytes(ctypes.byref(d), 8)
    assert a > 0 and b > a and a % 256 == 0
    # 4 batch-sized scratch planes of M*N*N or N*N complex64 grow linearly in B
    NN = 32 * 32
    assert b - a >= 4 * (2 * NN * 8 * 2 + NN * 8 * 2)
    assert L.ptycho_workspace_bytes(ctypes.byref(_dims(N=48)), 4) == 0     # unsupported N
    assert L.ptycho_workspace_bytes(ctypes.byref(_dims(M=17)), 4) == 0
    assert L.ptycho_workspace_bytes(ctypes.byref(_dims(H=32)), 4) == 0     # H < N + 1
    assert L.ptycho_workspace_bytes(ctypes.byref(d), 0) == 0
    assert L.ptycho_host_workspace_bytes(ctypes.byref(d), 4) > a


def test_multislice_workspace_keeps_one_mode_of_incident_waves_when_recomputing(L):
    from paper_2510_20929_gb300 import api
    N, M, S, B = 32, 3, 4, 8
    d = _dims(H=96, W=100, N=N, M=M, J=20)
    keep = L.ptycho_workspace_bytes_ms(ctypes.byref(d), ctypes.byref(api.make_multislice(S, 2e-6, 1e-10, 1e-8)), B)
    rec = L.ptycho_workspace_bytes_ms(ctypes.byref(d), ctypes.byref(api.make_multislice(S, 2e-6, 1e-10, 1e-8,
                                                                                        recompute=True)), B)
    # B (M - 1) (S - 1) N^2 complex64 fewer (up to the 256-byte alignment of the section)
    assert abs((keep - rec) - B * (M - 1) * (S - 1) * N * N * 8) < 256
    opts = api.make_opts(batch=B)
    keep_l = L.ptycho_workspace_bytes_lsqml_ms(ctypes.byref(d), ctypes.byref(api.make_multislice(S, 2e-6, 1e-10, 1e-8)),
                                               ctypes.byref(opts))
    rec_l = L.ptycho_workspace_bytes_lsqml_ms(
        ctypes.byref(d), ctypes.byref(api.make_multislice(S, 2e-6, 1e-10, 1e-8, recompute=True)), ctypes.byref(opts))
    assert keep_l - rec_l == keep - rec
    bad = api.make_multislice(S, 2e-6, 1e-10, 1e-8)
    bad.recompute = 2
    assert L.ptycho_workspace_bytes_ms(ctypes.byref(d), ctypes.byref(bad), B) == 0
    ws = ctypes.create_string_buffer(16)
    assert L.ptycho_forward_ms(ctypes.byref(d), ctypes.byref(bad), ws, ws, ws, ws, B, ws, 16, None) == 1   # ERR_ARG


def test_arguments_rejected_before_any_launch(L):
    from paper_2510_20929_gb300 import api
    P = ctypes.c_void_p
    fake = P(0x1000)      # never dereferenced: every call below fails its host checks first
    d = _dims()
    assert L.ptycho_forward(None, fake, fake, fake, fake, fake, 1 << 20, None) == 1
    assert L.ptycho_forward(ctypes.byref(_dims(N=48)), fake, fake, fake, fake, fake, 1 << 20, None) == 6
    assert L.ptycho_forward(ctypes.byref(d), P(0), fake, fake, fake, fake, 1 << 20, None) == 1
    assert L.ptycho_forward(ctypes.byref(d), fake, fake, fake, fake, P(0), 1 << 20, None) == 7
    assert L.ptycho_forward(ctypes.byref(d), fake, fake, fake, fake, P(0x1001), 1 << 20, None) == 7
    opts = api.make_opts(batch=0)
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                P(0), P(0), fake, 1 << 30, None) == 1
    opts = api.make_opts(batch=4)
    opts.precision = 7
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                P(0), P(0), fake, 1 << 30, None) == 1
    for bad in (dict(pos_step=-1.0), dict(pos_max_shift=float("nan"))):
        opts = api.make_opts(batch=4, update_positions=True, **bad)
        assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                    P(0), P(0), fake, 1 << 30, None) == 1
    opts = api.make_opts(batch=4)
    opts.object_per_epoch = 2
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                P(0), P(0), fake, 1 << 30, None) == 1
    # the per-epoch object accumulator needs H x W complex64 more workspace
    per_epoch = api.make_opts(batch=4, object_per_epoch=True)
    base = L.ptycho_workspace_bytes(ctypes.byref(d), 4)
    assert L.ptycho_workspace_bytes_opts(ctypes.byref(d), ctypes.byref(api.make_opts(batch=4))) == base
    assert L.ptycho_workspace_bytes_opts(ctypes.byref(d), ctypes.byref(per_epoch)) >= base + d.H * d.W * 8
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(per_epoch),
                                P(0), P(0), P(0x1000), base, None) == 7
    opts = api.make_opts(batch=4, noise=7)
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                P(0), P(0), fake, 1 << 30, None) == 1
    opts = api.make_opts(batch=4, delta_o=-1.0)
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                P(0), P(0), fake, 1 << 30, None) == 1
    opts = api.make_opts(batch=4)
    assert L.ptycho_lsqml_epoch(ctypes.byref(d), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                P(0), P(0), P(0x1000), 16, None) == 7           # workspace too small
    assert L.ptycho_adjoint(ctypes.byref(d), fake, fake, fake, fake, 9, 0.0, 4, fake, fake, P(0), P(0),
                            fake, 1 << 30, None) == 1                            # bad noise model
    assert L.ptycho_adjoint(ctypes.byref(d), fake, fake, fake, fake, 0, -1.0, 4, fake, fake, P(0), P(0),
                            fake, 1 << 30, None) == 1                            # negative eps
    assert L.ptycho_status_read(P(0), None) == 7
    assert L.ptycho_workspace_init(P(0x1001), 1 << 20, None) == 7
    # the split-BF16 DFT-GEMM precision: windows 32, 64, 128 only, an unknown precision is an argument error
    tc = api.make_opts(batch=4, precision="bf16x3")
    d256 = _dims(H=300, W=300, N=256)
    assert L.ptycho_lsqml_epoch(ctypes.byref(d256), fake, fake, fake, fake, P(0), ctypes.byref(tc),
                                P(0), P(0), fake, 1 << 30, None) == 6
    assert L.ptycho_forward_ex(ctypes.byref(_dims(N=16)), 1, 4, fake, fake, fake, fake, fake, 1 << 30, None) == 6
    assert L.ptycho_forward_ex(ctypes.byref(d), 2, 4, fake, fake, fake, fake, fake, 1 << 30, None) == 1
    assert L.ptycho_forward_ex(ctypes.byref(d), 1, 0, fake, fake, fake, fake, fake, 1 << 30, None) == 1
    assert L.ptycho_forward_ex(ctypes.byref(d), 1, 4, fake, fake, fake, fake, P(0x1000), 4096, None) == 7
    assert L.ptycho_adjoint_ex(ctypes.byref(d256), 1, fake, fake, fake, fake, 0, 0.0, 4, fake, fake, P(0), P(0),
                               fake, 1 << 30, None) == 6
    # BF16X3 reads the measured intensities with tensor copies: 16-byte aligned
    assert L.ptycho_adjoint_ex(ctypes.byref(d), 1, fake, fake, fake, P(0x100008), 0, 0.0, 4, fake, fake, P(0), P(0),
                               fake, 1 << 30, None) == 1
    # the relaxed-probe epoch takes FP32 only
    opr = api.make_opr_opts(2)
    assert L.ptycho_lsqml_epoch_opr(ctypes.byref(d), ctypes.byref(opr), fake, fake, fake, fake, fake, fake,
                                    P(0), ctypes.byref(tc), P(0), P(0), fake, 1 << 30, None) == 6


def test_binding_refuses_cpu_tensors():
    import torch
    from paper_2510_20929_gb300 import api
    obj = torch.zeros(64, 64, dtype=torch.complex64)
    probe = torch.zeros(1, 32, 32, dtype=torch.complex64)
    pos = torch.zeros(3, 2)
    with pytest.raises(ValueError):
        api.forward(obj, probe, pos)


def test_allocation_free_epoch_rejects_arguments_like_the_workspace_epoch(L):
    # same statuses as ptycho_lsqml_epoch, all returned by host checks before the
    # array's address is looked up (so no device is touched)
    from paper_2510_20929_gb300 import api
    P = ctypes.c_void_p
    fake = P(0x1000)
    opts = api.make_opts(batch=4)
    for dims, want in ((_dims(N=48), 6), (_dims(M=17), 6), (_dims(H=32), 1)):
        got_ws = L.ptycho_lsqml_epoch(ctypes.byref(dims), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                      P(0), P(0), fake, 1 << 30, None)
        got_static = L.ptycho_lsqml_epoch_static(ctypes.byref(dims), fake, fake, fake, fake, P(0),
                                                 ctypes.byref(opts), P(0), P(0), None)
        assert got_static == got_ws == want
    bad = api.make_opts(batch=4, noise=7)
    assert L.ptycho_lsqml_epoch_static(ctypes.byref(_dims()), fake, fake, fake, fake, P(0), ctypes.byref(bad),
                                       P(0), P(0), None) == 1
    assert L.ptycho_lsqml_epoch_static(None, fake, fake, fake, fake, P(0), ctypes.byref(opts), P(0), P(0),
                                       None) == 1
    big = _dims(H=8192, W=8192, N=128, M=5, J=100)
    assert L.ptycho_lsqml_epoch_static(ctypes.byref(big), fake, fake, fake, fake, P(0), ctypes.byref(opts),
                                       P(0), P(0), None) == 8


def test_tuning_set_rejects_unknown_variants(L):
    from paper_2510_20929_gb300 import api
    for dims, v in ((_dims(N=128, H=300, W=300), (3, 0, 0)), (_dims(N=64, H=100, W=100), (2, 0, 0)),
                    (_dims(), (0, 4, 0)), (_dims(N=256, H=300, W=300), (0, 2, 0)), (_dims(), (0, 0, 4)),
                    (_dims(), (-1, 0, 0))):
        arr = (ctypes.c_int32 * 3)(*v)
        assert L.ptycho_tuning_set(ctypes.byref(dims), 4, arr) == 1
    assert L.ptycho_tuning_set(ctypes.byref(_dims(N=48)), 4, (ctypes.c_int32 * 3)(0, 0, 0)) == 6
    assert L.ptycho_tuning_set(ctypes.byref(_dims()), 0, (ctypes.c_int32 * 3)(0, 0, 0)) == 1
