"""The C oracle under AddressSanitizer and UBSan: every entry point over odd shapes
(extents 1 and 2, ragged sizes) reads and writes only inside its exact-size arrays."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oracle_clean_under_sanitizers(tmp_path):
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not available")
    exe = tmp_path / "oracle_sanitize"
    build = subprocess.run(
        [cc, "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
         "-fno-omit-frame-pointer", "-ffp-contract=off", "-o", str(exe),
         os.path.join(HERE, "oracle_sanitize_driver.c"), os.path.join(ROOT, "oracle", "cdi_oracle.c"), "-lm"],
        capture_output=True, text=True)
    if build.returncode != 0:
        pytest.skip("no sanitizer runtime: " + build.stderr.strip().splitlines()[-1][:200])
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    assert "nonzero returns: 0" in run.stdout
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
