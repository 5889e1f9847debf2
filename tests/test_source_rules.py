"""Static checks on the native sources: portability to the Arm host and GPU-safety forms.

The library and the oracle must build the same way on x86 and Arm hosts, so:
  - no x86 intrinsics headers;
  - no -march=native in any build command;
  - the kernels compile for sm_103a alone.
The device code must never end a wait by faulting, so:
  - no trap instruction and no failing device assert;
  - no NVLink multicast or multimem forms, since the library is one process
    on one GPU.
  - every mbarrier wait is bounded by a timer, after which the kernel records an
    error and returns.
"""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources():
    pats = ["paper_2204_14194_gb300/csrc/*", "oracle/*.c", "oracle/*.py", "include/*.h",
            "paper_2204_14194_gb300/*.py", "__graft_entry__.py", "bench.py"]
    for p in pats:
        for f in glob.glob(os.path.join(ROOT, p)):
            if os.path.isfile(f):
                with open(f, errors="replace") as fh:
                    yield os.path.relpath(f, ROOT), fh.read()


def test_no_x86_specific_code_or_native_tuning():
    for name, text in _sources():
        assert not re.search(r"#\s*include\s*<(x86intrin|immintrin|emmintrin|xmmintrin)\.h>", text), name
        assert "-march=native" not in text and "-mtune=native" not in text, name


def test_device_code_has_no_trap_assert_or_multicast():
    for name, text in _sources():
        if not name.endswith((".cu", ".cuh")):
            continue
        code = re.sub(r"//[^\n]*", "", text)          # comments may describe what is avoided
        assert "__trap" not in code and not re.search(r"\btrap;", code), name
        assert not re.search(r"\bassert\s*\(", code), name
        assert "multimem" not in code and ".multicast" not in code, name


def test_kernels_build_for_sm103a_only():
    with open(os.path.join(ROOT, "paper_2204_14194_gb300", "build.py")) as f:
        text = f.read()
    assert re.findall(r"arch=compute_\w+,code=sm_\w+", text) == ["arch=compute_103a,code=sm_103a"]


def test_every_mbarrier_wait_goes_through_a_bounded_helper():
    """mbarrier.try_wait appears only inside the two wait helpers, and both give up after a
    %globaltimer limit; the raw try helper is called only by its bounded wait loop."""
    found = {}
    for name, text in _sources():
        n = text.count("mbarrier.try_wait")
        if n:
            found[os.path.basename(name)] = n
    assert found == {"k_device.cuh": 1, "k_gemm_tc.cu": 1}, found
    for name, text in _sources():
        if name.endswith(".cuh") and "mbarrier.try_wait" in text:
            body = text[text.index("bool bar_wait("):]
            body = body[:body.index("\n}\n")]
            assert "%%globaltimer" in body and "return false" in body
        if name.endswith("k_gemm_tc.cu"):
            body = text[text.index("bool mbar_wait("):]
            body = body[:body.index("\n}\n")]
            assert "gtimer()" in body and "return false" in body
            assert len(re.findall(r"\bmbar_try\(", text)) == 3      # definition + two calls in mbar_wait
            assert len(re.findall(r"\bmbar_try\(", body)) == 2
