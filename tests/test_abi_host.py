"""Host-only checks of the C ABI: the library builds and loads, exports every
symbol include/*.h declares, and validates arguments before any CUDA call
(smrt_create and the option setters touch no device, so these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2409_01076_gb300 as S
from paper_2409_01076_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names += re.findall(r"SMRT_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)
    return names


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "smrt_step" in names and "smrt_create" in names and len(names) >= 16
    lib = _lib.load()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding covers every one with the same name
    assert sorted(n for n, _, _ in _lib.SIGNATURES) == sorted(names)
    for n in names:
        assert callable(getattr(S, n)), n


def test_only_the_abi_is_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.path()], capture_output=True, text=True).stdout
    syms = [line.split()[-1] for line in out.splitlines() if line.strip()]
    assert syms and all(s.startswith("smrt_") for s in syms), syms[:10]


@pytest.mark.parametrize("args", [
    (1, 8, 0.7, 0.0, S.CAVITY),                    # nx < 2
    (8, 1, 0.7, 0.0, S.CAVITY),                    # ny < 2
    (8, 8, 0.5, 0.0, S.CAVITY),                    # tau must exceed 1/2
    (8, 8, float("nan"), 0.0, S.CAVITY),
    (8, 8, 0.7, 0.6, S.CAVITY),                    # |u_lid| >= 1/sqrt(3)
    (8, 8, 0.7, 0.0, S.bc_flags(0, 1, 1, 1)),      # unpaired periodic side
    (8, 8, 0.7, 0.0, S.bc_flags(1, 1, 3, 1)),      # kind 3 does not exist
    (8, 8, 0.7, 0.0, 1 << 9),                      # stray bits
    (1 << 20, 1 << 12, 0.7, 0.0, S.CAVITY),        # too large for one plane
])
def test_create_rejects_bad_arguments(args):
    with pytest.raises(S.SmrtError) as ei:
        S.smrt_create(*args)
    assert ei.value.status == S.SMRT_ERR_ARG
    assert "smrt_create" in str(ei.value)


def test_options_before_first_use():
    h = S.smrt_create(16, 12, 0.7, 0.05, S.CAVITY)
    assert S.smrt_time(h) == 0 and S.smrt_device_bytes(h) == 0
    S.smrt_set_option(h, S.SMRT_OPT_PRECISION, S.SMRT_PREC_F32)
    S.smrt_set_option(h, S.SMRT_OPT_LAYOUT, S.SMRT_LAYOUT_AA)
    S.smrt_set_option(h, S.SMRT_OPT_COLLISION, S.SMRT_COLLISION_TWO_TAU)
    S.smrt_set_option(h, S.SMRT_OPT_TAU_S, 0.9)
    S.smrt_set_option(h, S.SMRT_OPT_MEM_LIMIT, 1 << 20)
    assert S.smrt_get_option(h, S.SMRT_OPT_PRECISION) == S.SMRT_PREC_F32
    assert S.smrt_get_option(h, S.SMRT_OPT_TAU_S) == 0.9
    assert S.smrt_get_option(h, S.SMRT_OPT_ROUNDING) == S.SMRT_ROUND_NEAREST
    S.smrt_set_option(h, S.SMRT_OPT_ROUNDING, S.SMRT_ROUND_STOCHASTIC)
    assert S.smrt_get_option(h, S.SMRT_OPT_ROUNDING) == S.SMRT_ROUND_STOCHASTIC
    for key, val in [(S.SMRT_OPT_TAU_S, 0.5), (S.SMRT_OPT_TAU, -1.0), (S.SMRT_OPT_COLLISION, 7),
                     (S.SMRT_OPT_LAYOUT, 2), (S.SMRT_OPT_PRECISION, 9), (S.SMRT_OPT_CHECK_DIVERGENCE, 0.5),
                     (S.SMRT_OPT_ROUNDING, 2), (S.SMRT_OPT_ROUNDING, 0.5), (999, 0.0)]:
        with pytest.raises(S.SmrtError) as ei:
            S.smrt_set_option(h, key, val)
        assert ei.value.status == S.SMRT_ERR_ARG
    with pytest.raises(S.SmrtError):
        S.smrt_set_time(h, -1)
    S.smrt_set_time(h, 4)
    assert S.smrt_time(h) == 4
    S.smrt_destroy(h)


def test_null_handle_is_rejected():
    lib = _lib.load()
    assert lib.smrt_step(None, 1) == S.SMRT_ERR_ARG
    assert lib.smrt_time(None) == -1
    assert lib.smrt_device_bytes(None) == 0
    lib.smrt_destroy(None)
    out = ctypes.c_void_p(1)
    assert lib.smrt_create(0, 0, 0.7, 0.0, 0, ctypes.byref(out)) == S.SMRT_ERR_ARG
    assert out.value is None


# The TMA-convolution and fused element-wise entry points check their arguments before any CUDA
# call: each of these is rejected with SMRT_ERR_ARG and a message naming the function (no GPU needed).
_BAD_NN_CALLS = [
    ("smrt_nn_conv3_tma", (None, 1, 4, 4, 24, None, 8, 1.0, 0.0, None, 8, None, None)),
    ("smrt_nn_conv3_tma_bias_act", (None, 1, 4, 4, 16, None, 12, None, 1, None, None, None, None, None)),
    ("smrt_nn_conv3_wgrad_tma", (None, 1, 4, 4, 16, None, 12, 1.0, None, 144, None, None)),
    ("smrt_nn_pack3", (None, 8, 24, None, None)),
    ("smrt_nn_to_half_blocked", (None, 1, 4, 4, 12, 1.0, None, None)),
    ("smrt_nn_to_half_blocked_pad", (None, 1, 4, 4, 3, 12, 1.0, None, None)),
    ("smrt_nn_pad3", (None, 8, 3, 2, None, None)),
    ("smrt_nn_unpad3_add", (None, 8, 3, 16, None, None)),
    ("smrt_nn_bias_act_blocked", (None, None, 1, 4, 4, 12, 1, None, None, None, None)),
    ("smrt_nn_bias_act_bwd_blocked", (None, None, 1, 4, 4, 12, 1, None, None, None, None)),
    ("smrt_nn_avgpool2_blocked", (None, 1, 3, 4, 8, None, None, None)),
    ("smrt_nn_upcat", (None, 1, 2, 2, 12, None, 8, None, None, None)),
    ("smrt_nn_upcat_bwd", (None, 1, 2, 2, 6, 4, None, None, None)),
    ("smrt_nn_conv1x1_small", (None, 16, 32, None, None, 4, None, None)),
    ("smrt_nn_conv1x1_small_bwd", (None, None, 16, 32, None, 3, None, None, None, None)),
]


@pytest.mark.parametrize("name,args", _BAD_NN_CALLS, ids=[c[0] for c in _BAD_NN_CALLS])
def test_nn_entry_points_reject_bad_arguments_on_the_host(name, args):
    rc = getattr(_lib.load(), name)(*args)
    assert rc == S.SMRT_ERR_ARG, (name, rc)
    assert name in S.smrt_last_error(None)


def test_pack3_halves_rejects_narrow_chunks():
    assert S.smrt_nn_pack3_halves(8, 24) == -1 and S.smrt_nn_pack3_halves(0, 32) == -1
    assert S.smrt_nn_pack3_halves(130, 32) == 9 * 32 * 256
