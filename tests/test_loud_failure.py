"""The product path has no fallback: without libnegf.so the package refuses
to import (checked on a copy of the package without the library)."""
import os
import shutil
import subprocess
import sys


def test_import_without_the_library_raises(tmp_path):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = os.path.join(root, "paper_2605_19910_gb300")
    dst = tmp_path / "paper_2605_19910_gb300"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "*.so.arch", "_build", "__pycache__"))
    code = "import paper_2605_19910_gb300"
    r = subprocess.run([sys.executable, "-c", code], cwd=str(tmp_path), capture_output=True, text=True,
                       env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0
    assert "libnegf.so not found" in r.stderr
