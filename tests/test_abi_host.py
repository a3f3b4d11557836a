"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/llb.h declares, validates arguments before touching
the device, and its storage accounting reproduces the array counts the paper
prints (Sec. III A and III C)."""
import json
import os
import re

import pytest

from paper_2301_01622_gb300 import llb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib_or_skip():
    if not os.path.exists(llb.LIB_PATH):
        pytest.skip("libllb.so not built")
    return llb.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "llb.h")).read()
    return sorted(set(re.findall(r"LLB_API\s+[\w\s\*]+?\b(llb_\w+)\s*\(", text)))


def test_header_declares_and_library_exports_every_symbol():
    L = _lib_or_skip()
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/llb.h but not exported"
    assert sorted(llb.exported_symbols()) == names


def test_params_defaults():
    _lib_or_skip()
    p = llb.llb_params_default()
    assert (p.ncomp, p.storage, p.scheme, p.kernel) == (1, llb.LLB_F32, llb.LLB_SCHEME_MOMENT, llb.LLB_KERNEL_AUTO)
    assert p.beta == 0.7 and p.A_s == 0.01 and p.A_h == 0.0 and p.h_c == 3
    assert p.stream is None and p.buffers[0] is None


def test_storage_accounting_matches_paper():
    """20 vs 38 arrays (one component, D3Q19) and 22 vs 76 (two components)."""
    _lib_or_skip()
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_counts.json")))
    mom1 = llb.llb_footprint_query(128, 128, 128, 19, llb.llb_params_default())
    pop1 = llb.llb_footprint_query(128, 128, 128, 19, llb.llb_params_default(scheme=llb.LLB_SCHEME_POPULATION))
    mom2 = llb.llb_footprint_query(128, 128, 128, 19, llb.llb_params_default(ncomp=2))
    pop2 = llb.llb_footprint_query(128, 128, 128, 19,
                                   llb.llb_params_default(ncomp=2, scheme=llb.LLB_SCHEME_POPULATION))
    assert mom1.arrays == g["hydro_arrays_one_component_flipflop"]["value"]
    assert pop1.arrays == g["population_arrays_d3q19_one_component_flipflop"]["value"]
    assert mom2.arrays == g["hydro_arrays_two_component_flipflop"]["value"]
    assert pop2.arrays == g["population_arrays_d3q19_two_component_flipflop"]["value"]
    # the streaming step of the two-component D3Q19 scheme reads 11 fields at
    # 18 neighbours: 198 values, 792 bytes in FP32 (Sec. IV A)
    assert mom2.fields * 18 == g["stream_reads_two_component_d3q19"]["value"]
    assert mom2.fields * 18 * 4 == g["stream_read_bytes_fp32_two_component_d3q19"]["value"]
    # bytes per node and state size (FP32)
    assert mom1.bytes_per_node == 80 and pop1.bytes_per_node == 152
    # one state copy: 10 FP32 fields per node plus periodic ghost rows/columns; the
    # one-component FP32 state rounds its rows up to whole 32-node blocks
    assert 10 * 4 * 128 ** 3 <= mom1.state_bytes == 10 * 4 * 160 * 130 * 128
    assert pop1.state_bytes == 19 * 4 * 128 ** 3
    q27 = llb.llb_footprint_query(8, 8, 8, 27, llb.llb_params_default(scheme=llb.LLB_SCHEME_POPULATION))
    assert q27.bytes_per_node == 216
    f64 = llb.llb_footprint_query(8, 8, 8, 27, llb.llb_params_default(storage=llb.LLB_F64))
    assert f64.bytes_per_node == 160
    assert llb.llb_state_bytes(8, 8, 8, 19) == 10 * 4 * 32 * 10 * 8
    # other states keep rows rounded to 8 nodes (FP64: 8 + 16 ghost columns)
    assert llb.llb_state_bytes(8, 8, 8, 19, llb.llb_params_default(storage=llb.LLB_F64)) == 10 * 8 * 24 * 10 * 8


@pytest.mark.parametrize("args", [
    (0, 8, 8, 19, 0.8), (8, -1, 8, 19, 0.8), (8, 8, 8, 15, 0.8), (8, 8, 8, 19, 0.5), (8, 8, 8, 19, float("nan")),
])
def test_create_rejects_bad_arguments_without_device(args):
    _lib_or_skip()
    with pytest.raises(llb.LLBError) as e:
        llb.llb_create(*args)
    assert e.value.status == llb.LLB_EINVAL


def test_bad_params_rejected():
    _lib_or_skip()
    for kw in ({"ncomp": 3}, {"storage": 7}, {"scheme": 9}, {"kernel": 7}):
        with pytest.raises(llb.LLBError) as e:
            llb.llb_footprint_query(8, 8, 8, 19, llb.llb_params_default(**kw))
        assert e.value.status == llb.LLB_EINVAL


def test_null_context_calls_fail_cleanly():
    L = _lib_or_skip()
    assert L.llb_step(None, 1) == llb.LLB_EINVAL
    assert L.llb_synchronize(None) == llb.LLB_EINVAL
    L.llb_destroy(None)  # NULL-safe
    assert llb.status_string(llb.LLB_EUNSTABLE).startswith("unstable")


def test_checked_build_exports_the_same_symbols_and_reports_itself():
    """libllb_checked.so (built with -DLLB_CHECKED) exports every declared
    function; llb_checked_status reports enabled = 1 there and 0 in libllb.so
    (*enabled is set before the device synchronisation, so no GPU is needed)."""
    import ctypes as C

    from paper_2301_01622_gb300 import build as B
    if not (os.path.exists(B.LIB) and os.path.exists(B.LIB_CHECKED)):
        pytest.skip("libraries not built")
    for path, want in ((B.LIB, 0), (B.LIB_CHECKED, 1)):
        L = C.CDLL(path)
        for n in _declared():
            assert hasattr(L, n), f"{n} not exported by {os.path.basename(path)}"
        en, site, idx = C.c_int(-1), C.c_int(-1), C.c_longlong(-1)
        L.llb_checked_status.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
        L.llb_checked_status(C.byref(en), C.byref(site), C.byref(idx))
        assert en.value == want
        assert site.value == 0 and idx.value == 0
