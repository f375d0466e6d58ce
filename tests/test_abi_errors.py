"""Every status-returning entry point of the C ABI refuses null handles and
pointers with an error status and a message, before it touches the GPU, so
this runs on the CPU.  The entry points are function-try-blocks (no C++
exception crosses the ABI); this checks that their ordinary error returns
pass through unchanged."""
import ctypes as C

import pytest

# entry points that do not return a gs_status
NOT_STATUS = {"gs_version", "gs_build_flags", "gs_last_error", "gs_ctx_bytes", "gs_destroy", "gs_mesh_destroy",
              "gs_batch_destroy", "gs_server_destroy", "gs_raster_destroy", "gs_rigid_destroy", "gs_result_free"}
# a null context for profiling reads as "profiling is off"
EXPECTED = {"gs_profile_read": "GS_ESTATE"}


def _null_args(argtypes):
    args = []
    for t in argtypes:
        if t in (C.c_float, C.c_double):
            args.append(0.0)
        elif t in (C.c_int, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64, C.c_size_t, C.c_long, C.c_ulong):
            args.append(0)
        else:  # pointers and handles
            args.append(None)
    return args


@pytest.fixture(scope="module")
def gs():
    from paper_2104_02646_gb300 import gradsim
    gradsim.load(build=True)
    return gradsim


def test_null_arguments_give_an_error_and_a_message(gs):
    L = gs.load()
    checked = []
    for name, (restype, argtypes) in sorted(gs._PROTOS.items()):
        if name in NOT_STATUS:
            continue
        fn = getattr(L, name)
        st = fn(*_null_args(argtypes))
        want = getattr(gs, EXPECTED.get(name, "GS_EINVAL"))
        assert st == want, (name, st)
        msg = L.gs_last_error().decode()
        assert msg, name
        checked.append(name)
    assert len(checked) >= 35


def test_error_codes_match_the_header(gs):
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "include", "gradsim.h")).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"\b(GS_[EW]\w+|GS_OK|GS_PENDING)\s*=\s*(-?\d+)", src))
    assert codes["GS_EINTERNAL"] == -11
    for k, v in codes.items():
        assert getattr(gs, k) == v, k
