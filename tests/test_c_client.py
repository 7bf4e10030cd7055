"""The boundary is a C ABI: a C99 client compiled against include/irk.h (gcc, no C++), linked to
libirk.so, calls the host-only entry points (CPU, no device).  Expected values are the Q = 2
Radau IIA closed forms (tests/golden/radau_iia_closed_forms.txt) and the documented defaults."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CLIENT = r"""
#include <stdio.h>
#include "irk.h"

int main(void) {
  irk_options o;
  double A[4], b[2], c[2];
  irk_default_options(&o);
  printf("rtol %.3e restart %d mg %d graph %d\n", o.rtol, o.restart, o.mg_precision, o.use_graph);
  if (irk_tableau_factors(2, 0, A) != IRK_OK || irk_tableau_factors(2, 1, b) != IRK_OK ||
      irk_tableau_factors(2, 2, c) != IRK_OK)
    return 2;
  printf("A %.17g %.17g %.17g %.17g\n", A[0], A[1], A[2], A[3]);
  printf("b %.17g %.17g c %.17g %.17g\n", b[0], b[1], c[0], c[1]);
  printf("einval %d %s\n", (int)irk_tableau_factors(0, 0, A), irk_strerror(IRK_EINVAL) != NULL ? "msg" : "null");
  printf("ndofs %ld\n", (long)irk_ndofs(NULL));
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib_dir():
    from tests.test_capi_load import _built_lib
    capi = _built_lib()
    return os.path.dirname(capi.LIB_PATH)


def test_c99_client_links_and_calls_the_library(tmp_path, lib_dir):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(CLIENT)
    exe = tmp_path / "client"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", lib_dir, "-lirk", "-Wl,-rpath," + lib_dir],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    lines = dict(l.split(" ", 1) for l in r.stdout.strip().splitlines())
    assert lines["rtol"] == "1.000e-10 restart 30 mg 0 graph 1"   # mg 0: precision chosen at create
    A = [float(x) for x in lines["A"].split()]
    assert max(abs(a - e) for a, e in zip(A, [5 / 12, -1 / 12, 3 / 4, 1 / 4])) < 1e-15
    bc = lines["b"].split()
    assert abs(float(bc[0]) - 0.75) < 1e-15 and abs(float(bc[1]) - 0.25) < 1e-15
    assert abs(float(bc[3]) - 1 / 3) < 1e-15 and abs(float(bc[4]) - 1.0) < 1e-15
    assert lines["einval"] == "-1 msg"
    assert lines["ndofs"] == "-1"
