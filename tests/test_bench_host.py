"""CPU tests of the benchmark's host logic: the source hash that decides whether a stored
ncu traffic figure still applies, the traffic rule itself, and the parsing of the clock
samples taken during the timed region (a run with a slowdown reason must show it)."""
import os
import tempfile

import bench


def test_code_without_comments_keeps_code_and_strings():
    a = 'int f() { // a comment\n  return 1; /* block\n comment */ }\nconst char* s = "// not a comment";\n'
    b = 'int f() {\n  return 1;   }\n// another\nconst char* s = "// not a comment";'
    assert bench.code_without_comments(a) == bench.code_without_comments(b)
    assert '"//notacomment"' in bench.code_without_comments(a).replace(" ", "")
    assert bench.code_without_comments("x = 1;") != bench.code_without_comments("x = 2;")


def test_traffic_applies_only_to_the_captured_build_and_shape(monkeypatch):
    c = bench.TRAFFIC_CAPTURE
    info = {"table2_bytes": c["table2_bytes"], "table3_bytes": c["table3_bytes"]}
    shape = dict(c["shape"], chunk=12345, grid=304)  # other shape keys do not matter
    monkeypatch.setattr(bench, "library_sources_sha", lambda: c["sources_sha256"])
    n = 3_000_000_000
    assert bench.measured_traffic("genome", n, shape, info) == int(round(c["bytes_per_base"] * n))
    assert bench.measured_traffic("chromosome", n, shape, info) is None
    assert bench.measured_traffic("genome", n, dict(shape, threads=1024), info) is None
    assert bench.measured_traffic("genome", n, shape, dict(info, table3_bytes=0)) is None
    monkeypatch.setattr(bench, "library_sources_sha", lambda: "0" * 64)
    assert bench.measured_traffic("genome", n, shape, info) is None


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _clocks_from(lines):
    c = bench.Clocks(0)
    fd, c.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    c.proc = _FakeProc()
    return c.stop()


def test_clock_samples_give_median_max_and_reasons():
    ok = "0, {sm}, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, {cap}"
    r = _clocks_from([ok.format(sm=2070, cap="Not Active"), ok.format(sm=2055, cap="Not Active"),
                      ok.format(sm=2070, cap="Active"), "garbage line"])
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    hot = "0, 1500, 2070, 900.0, 0x40, Not Active, Active, Not Active, Not Active"
    assert _clocks_from([hot])["reasons"] == ["hw_thermal_slowdown"]
    assert _clocks_from([])["reasons"] == ["no samples"]
