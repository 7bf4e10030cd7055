"""Without the compiled library the package has no CPU fallback: every entry point raises (CPU)."""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import paper_2209_06700_gb300 as p
calls = {
    "Solver": lambda: p.Solver(2, 4, 2, 2, 0.1),
    "tableau_factors": lambda: p.tableau_factors(2, "A"),
    "element_factors": lambda: p.element_factors(2, "Me"),
    "autotune_report": p.autotune_report,
}
for name, call in calls.items():
    try:
        call()
        print(name, "RAN")
    except OSError as e:
        print(name, "OSError", "libirk.so" in str(e))
"""


def test_every_entry_point_raises_without_the_library(tmp_path):
    pkg = tmp_path / "paper_2209_06700_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2209_06700_gb300"), pkg,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    assert not (pkg / "libirk.so").exists()
    r = subprocess.run([sys.executable, "-c", PROBE], cwd=tmp_path, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 4 and all(l.endswith("OSError True") for l in lines), lines
