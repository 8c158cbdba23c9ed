"""The generated rational program (Sec. 3.3 Step 3 / Sec. 4.3.1) without a
GPU: rp_codegen_source writes one kernel's coefficient table, data-parameter
maps and grid dimensionality into the source exactly (the hexadecimal
constants read back to the same floats), and the source compiles for
sm_103a with NVRTC (which needs no GPU)."""
import ctypes as C
import re

import numpy as np
import pytest
import torch

import paper_1906_00142_gb300 as rp
import workloads as W


def host_program(prog):
    K = prog["aN"].shape[0]
    d = int(prog["d"])
    buf = torch.zeros(rp.rp_program_size(K, d), dtype=torch.uint8)
    aN, bN, gd, tab = rp.program_views(buf, K, d)
    aN.copy_(torch.from_numpy(prog["aN"]))
    bN.copy_(torch.from_numpy(prog["bN"]))
    gd.copy_(torch.from_numpy(prog["grid_dims"].astype(np.int32)))
    tab.copy_(torch.from_numpy(prog["table"]))
    return buf


def _floats(src, name):
    body = src[src.index(name + "["):]
    body = body[body.index("{") + 1:body.index("}")]
    return np.array([float.fromhex(t.strip()[:-1]) for t in body.split(",") if t.strip()],
                    np.float32)


@pytest.fixture(scope="module")
def generated():
    rp.load_library()
    prog = W.synthetic_program(3, 3, seed=5)
    prog["table"][2, 7, 4, 1, 0] = 2.0 ** -140          # a subnormal survives the round trip
    return prog, rp.rp_codegen_source(host_program(prog), 3, 3, 2)


def test_generated_source_holds_the_program_exactly(generated):
    prog, src = generated
    np.testing.assert_array_equal(_floats(src, "g_tab"), prog["table"][2].reshape(-1))
    ab = _floats(src, "g_ab")
    np.testing.assert_array_equal(ab[:8], prog["aN"][2])
    np.testing.assert_array_equal(ab[8:], prog["bN"][2])
    assert f"g_ab + kNmet, {int(prog['grid_dims'][2])}, s)" in src
    assert "__float_as_int(q1.w) == 2;" in src
    assert "eval_cfg<4, true>" in src
    # architecture constants of the default rp_hw_fixed
    assert "const HwC hw = {32, 64, 65536, 58368, " in src
    # size query and a too-small buffer
    lib = rp.load_library()
    buf = host_program(prog)
    n = C.c_size_t(10)
    h = rp.hw_struct()
    small = C.create_string_buffer(10)
    assert lib.rp_codegen_source(C.c_void_p(buf.data_ptr()), 3, 3, 2, C.byref(h), small, C.byref(n)) == -3
    assert n.value == len(src) + 1
    assert lib.rp_codegen_source(C.c_void_p(buf.data_ptr()), 3, 3, 3, C.byref(h), None, C.byref(n)) == -1


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    return None


def test_generated_source_compiles_for_sm_103a(generated):
    _, src = generated
    nv = _nvrtc()
    if nv is None:
        pytest.skip("NVRTC not found")
    prog = C.c_void_p()
    assert nv.nvrtcCreateProgram(C.byref(prog), src.encode(), b"rp_generated.cu", 0, None, None) == 0
    opts = (C.c_char_p * 2)(b"--gpu-architecture=sm_103a", b"-std=c++17")
    rc = nv.nvrtcCompileProgram(prog, 2, opts)
    n = C.c_size_t(0)
    nv.nvrtcGetProgramLogSize(prog, C.byref(n))
    log = C.create_string_buffer(n.value + 1)
    nv.nvrtcGetProgramLog(prog, log)
    assert rc == 0, log.value.decode()[:3000]
    nv.nvrtcGetCUBINSize(prog, C.byref(n))
    assert n.value > 0
    nv.nvrtcDestroyProgram(C.byref(prog))
