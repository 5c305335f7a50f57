"""CPU checks of the measurement tooling: the traffic stamp ignores comments but not code, and the
ncu summary reads a launch list and a traffic capture into the expected figures."""

import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load(name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(ROOT, name + ".py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_code_only_drops_comments_keeps_code():
    b = _load("bench")
    a = "int x = 1; // one\n/* block\n comment */ int y = 2;\n"
    assert b._code_only(a) == b._code_only("int x = 1;\n\n  int y = 2;")
    assert b._code_only(a) != b._code_only("int x = 2; int y = 2;")
    assert len(b.source_sha()) == 16


HEADER = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size","Grid Size",' \
         '"Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n'


def _row(i, kernel, metric, unit, value):
    return '"%d","1","python","h","%s","1","7","(256, 1, 1)","(152, 1, 1)","0","10.3","s","%s","%s","%s"\n' % (
        i, kernel, metric, unit, value)


def test_ncu_summary_launches_and_traffic(tmp_path):
    s = _load("ncu_summary")
    log = tmp_path / "l.csv"
    log.write_text("==PROF== noise\n" + HEADER +
                   _row(0, "void fftenkf::col_fused_kernel<4096, 16, 2, 0>(ColFusedParams)", "gpu__time_duration.sum", "ns", "3,000") +
                   _row(1, "void fftenkf::row_inv_kernel<2048, 16, 1>(RowInvParams)", "gpu__time_duration.sum", "ns", "1,000") +
                   _row(2, "void at::elementwise_kernel<int>()", "gpu__time_duration.sum", "ns", "9,999"))
    table = s.launches(str(log))
    assert "`col_fused_kernel<4096, 16, 2, 0>` | 1 | 3 | 3 | 75.0%" in table
    assert "elementwise" not in table
    b = _load("bench")
    small = b.pass_bytes(64, 64, 4, 4, 2, 2)["row_inv"]
    dram = tmp_path / "d.csv"
    dram.write_text(HEADER +
                    _row(5, "void fftenkf::row_inv_kernel<32, 16, 1>(RowInvParams)", "dram__bytes_read.sum", "byte", "%d" % (small // 2)) +
                    _row(5, "void fftenkf::row_inv_kernel<32, 16, 1>(RowInvParams)", "dram__bytes_write.sum", "byte", "%d" % (small // 2)) +
                    _row(5, "void fftenkf::row_inv_kernel<32, 16, 1>(RowInvParams)", "gpu__time_duration.sum", "ns", "1000"))
    _, js = s.traffic([str(dram)], 64, 64, 4, 2, 2, 4, 20, "abc")
    full = b.pass_bytes(64, 64, 4, 20, 2, 2)["row_inv"]
    assert js["row_inv"]["source_sha"] == "abc"
    assert abs(js["row_inv"]["dram_bytes_per_launch_full"] - full) <= 1e-6 * full
