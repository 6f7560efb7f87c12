"""Launch-shape table of the library (vca_tune_*), host side only: entries, lookup keys, the file
form, and the environment variable that preloads a table."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vca():
    from paper_2304_12384_gb300 import build
    build.build()
    from paper_2304_12384_gb300 import vca as v
    v.lib()
    yield v
    v.vca_tune_clear()


ENTRY = dict(width=640, height=360, bit_depth=8, block_size=32, low_pass=1, chroma_format=0, kernel=1,
             plain_warps=8, tc_ctas=0, ms_per_frame=0.25)


def test_set_lookup_and_keys(vca):
    vca.vca_tune_clear()
    cfg = vca._config(640, 360, 8, 32, True)
    assert vca.vca_tune_lookup(cfg) is None
    vca.vca_tune_set(**ENTRY)
    got = vca.vca_tune_lookup(cfg)
    assert got["plain_warps"] == 8 and got["kernel"] == 1 and abs(got["ms_per_frame"] - 0.25) < 1e-7
    # kernel selector and max_batch are not part of the key; the other fields are
    assert vca.vca_tune_lookup(vca._config(640, 360, 8, 32, True, kernel=2, max_batch=7))["plain_warps"] == 8
    for other in (vca._config(640, 360, 10, 32, True), vca._config(640, 360, 8, 16, True),
                  vca._config(640, 360, 8, 32, False), vca._config(640, 352, 8, 32, True)):
        assert vca.vca_tune_lookup(other) is None
    # replacing, not duplicating
    vca.vca_tune_set(**dict(ENTRY, plain_warps=2))
    assert vca.vca_tune_lookup(cfg)["plain_warps"] == 2
    vca.vca_tune_clear()
    assert vca.vca_tune_lookup(cfg) is None


@pytest.mark.parametrize("bad", [dict(plain_warps=3), dict(kernel=0), dict(tc_ctas=-1), dict(block_size=24),
                                 dict(width=0)])
def test_bad_entries_are_rejected(vca, bad):
    with pytest.raises(vca.VcaError) as ei:
        vca.vca_tune_set(**dict(ENTRY, **bad))
    assert ei.value.status == vca.VCA_E_ARG


def test_file_round_trip_and_malformed_files(vca, tmp_path):
    vca.vca_tune_clear()
    vca.vca_tune_set(**ENTRY)
    vca.vca_tune_set(**dict(ENTRY, width=3840, height=2160, kernel=2, tc_ctas=114, ms_per_frame=0.0042))
    path = tmp_path / "table.txt"
    vca.vca_tune_save(str(path))
    lines = [ln for ln in path.read_text().splitlines() if not ln.startswith("#")]
    assert len(lines) == 2
    vca.vca_tune_clear()
    vca.vca_tune_load(str(path))
    e = vca.vca_tune_lookup(vca._config(3840, 2160, 8, 32, True))
    assert e["kernel"] == 2 and e["tc_ctas"] == 114
    bad = tmp_path / "bad.txt"
    bad.write_text(path.read_text() + "640 360 8 32 1 0 1 5 0 0.1\n")  # 5 warps: not a shape
    with pytest.raises(vca.VcaError) as ei:
        vca.vca_tune_load(str(bad))
    assert ei.value.status == vca.VCA_E_ARG and "line" in str(ei.value)
    assert vca.vca_tune_lookup(vca._config(3840, 2160, 8, 32, True))["tc_ctas"] == 114  # unchanged
    with pytest.raises(vca.VcaError):
        vca.vca_tune_load(str(tmp_path / "missing.txt"))
    vca.vca_tune_clear()


def test_environment_variable_preloads_the_table(tmp_path):
    path = tmp_path / "env.txt"
    path.write_text("# comment\n1920 1080 10 32 1 0 2 4 76 0.003\n")
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2304_12384_gb300 import vca\n"
            "e = vca.vca_tune_lookup(vca._config(1920, 1080, 10, 32, True))\n"
            "print(e['tc_ctas'], e['kernel'])\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, VCA_TUNE_FILE=str(path)),
                         capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["76", "2"]
