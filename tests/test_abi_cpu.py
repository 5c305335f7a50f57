"""CPU checks of the library boundary: it builds, loads, exports every declared entry point,
and rejects bad dimensions before touching the GPU."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fftenkf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fftenkf_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1001_1588_gb300 import abi, build
    if not os.path.exists(abi.LIB_PATH):
        build.build()
    return abi.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1001_1588_gb300 import abi
    assert set(_declared()) <= set(abi.declared_symbols())


@pytest.mark.parametrize(
    "dims,status",
    [((64, 64, 1, 1), 2), ((64, 60, 1, 4), 2), ((80, 64, 1, 4), 2), ((64, 64, 17, 4), 2), ((0, 64, 1, 4), 1),
     ((64, 16384, 1, 4), 2), ((8192, 64, 1, 4), 2)],
)
def test_plan_rejects_bad_dims_without_gpu(lib, dims, status):
    from paper_1001_1588_gb300 import abi
    with pytest.raises(abi.FftEnkfError) as ei:
        abi.fftenkf_plan_create(*dims, abi.FFTENKF_F32, [1] * max(1, dims[2]))
    assert ei.value.status == status


def test_too_many_observed_blocks(lib):
    from paper_1001_1588_gb300 import abi
    with pytest.raises(abi.FftEnkfError) as ei:
        abi.fftenkf_plan_create(64, 64, 5, 4, abi.FFTENKF_F32, [1, 1, 1, 1, 1])
    assert ei.value.status == abi.FFTENKF_EUNSUPPORTED


def test_status_strings(lib):
    from paper_1001_1588_gb300 import abi
    assert abi.fftenkf_status_string(0) == "ok"
    assert "invalid" in abi.fftenkf_status_string(1)
    assert abi.fftenkf_pass_count() == 10
    assert abi.fftenkf_pass_name(2) == "col_stats"
    assert abi.fftenkf_pass_name(9) == "col_fused"


def test_missing_library_fails_loudly(monkeypatch):
    from paper_1001_1588_gb300 import abi
    monkeypatch.setattr(abi, "_lib", None)
    monkeypatch.setattr(abi, "LIB_PATH", "/nonexistent/libfftenkf.so")
    with pytest.raises(ImportError):
        abi.lib()


def test_pass_byte_model_matches_analysis_model():
    """The per-pass byte model of an analysis with an estimated spectrum adds up to the analysis
    byte model once the pass this design adds is taken out: the transposed copy of rhat (written
    once, read once more).  The anomaly rows take the first member as pivot, so there is no mean
    pass and no mean read."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    for (ny, nx, M, N, no, s) in [(4096, 4096, 4, 20, 2, 2), (512, 512, 3, 5, 1, 4)]:
        pb = b.pass_bytes(ny, nx, M, N, no, s)
        used = ["row_fwd_anomaly", "rhat_transpose", "col_stats", "row_fwd_innovation", "col_update", "row_inv"]
        extra = 2 * no * (nx // 2 + 1) * ny * 8
        tot = sum(pb[k] for k in used) - extra
        ref = b.analysis_bytes(ny, nx, M, N, no, s)
        assert abs(tot - ref) / ref < 0.005, (tot, ref)   # packed nx/2 vs nx/2+1 columns


# Morphing entry points: argument checks that return before any CUDA call (fake, aligned addresses).
def test_morph_rejects_before_launch(lib):
    plane = 8 * 8 * 4
    base = 0x1000000
    # residual blocks of ext (from base + 2*K*plane) alias u
    assert lib.fftenkf_morph_forward(base + 4 * plane, base + 100 * plane, base, 1, 2, 8, 8, 4, 0.0, None) == 1
    assert lib.fftenkf_morph_forward(base, base + 100 * plane, base + 10 * plane, 1, 2, 8, 8, 1025, 0.0, None) == 1
    assert lib.fftenkf_morph_forward(base, base + 100 * plane, base + 10 * plane, 0, 2, 8, 8, 4, 0.0, None) == 1
    assert lib.fftenkf_morph_forward(base + 2, base + 100 * plane, base + 10 * plane, 1, 2, 8, 8, 4, 0.0, None) == 1
    assert lib.fftenkf_morph_forward(None, base + 100 * plane, base + 10 * plane, 1, 2, 8, 8, 4, 0.0, None) == 1
    assert lib.fftenkf_morph_forward(base, base + 100 * plane, base + 10 * plane, 1, 2, 65536, 65536, 4, 0.0, None) == 2
    assert lib.fftenkf_morph_forward(base, base + 100 * plane, base + 10 * plane, 1, 2, 8, 8, 4, -1.0, None) == 1
    assert lib.fftenkf_morph_forward(base, base + 100 * plane, base + 10 * plane, 1, 2, 8, 8, 4, float("nan"), None) == 1
    assert lib.fftenkf_morph_reference(base, base + plane, 3, 2, 8, 8, None) == 1     # ext_ref inside ext
    assert lib.fftenkf_morph_reference(base, base + 100 * plane, 3, 0, 8, 8, None) == 1
    assert lib.fftenkf_morph_inverse(base, base + 100 * plane, base + plane, 1, 2, 8, 8, None) == 1   # u_out in ext
    assert lib.fftenkf_morph_inverse(base, base + 100 * plane, base + 100 * plane, 1, 2, 8, 8, None) == 1
