"""include/nao.h is a plain C header: a C11 program that includes it compiles with every warning
as an error, links against libnao.so and calls the entry points that need no GPU (options,
status strings, argument checks, the host-only partition and spline fit), from C rather than
through ctypes."""
import shutil
import subprocess
from pathlib import Path

import pytest

from paper_1912_06636_gb300 import nao

ROOT = Path(__file__).resolve().parents[1]

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "nao.h"

#define CHECK(c) do { if (!(c)) { printf("FAIL line %d: %s\n", __LINE__, #c); return 1; } } while (0)

int main(void) {
    nao_options o;
    CHECK(nao_default_options(&o) == NAO_OK);
    CHECK(o.max_batch_points == 200 && o.split_slices == 12);
    CHECK(strcmp(nao_status_string(NAO_OK), "ok") == 0);
    nao_grid *g = (nao_grid *)&o;
    CHECK(nao_grid_create(NULL, &o, &g) == NAO_ERR_INVALID_ARG && g == NULL);
    CHECK(nao_destroy(NULL) == NAO_OK);
    CHECK(strlen(nao_last_error()) > 0);

    /* five points on a line, B = 2: batches {1}, {3, 4}, {0, 2} by the bisection rule */
    const double xyz[15] = {3, 0, 0, 0, 0, 0, 4, 0, 0, 1, 0, 0, 2, 0, 0};
    int64_t off[4], perm[5], nbat = 0;
    CHECK(nao_partition_points(xyz, 5, 2, 3, off, perm, &nbat) == NAO_OK && nbat == 3);
    CHECK(off[0] == 0 && off[1] == 1 && off[2] == 3 && off[3] == 5);
    CHECK(perm[0] == 1 && perm[1] == 3 && perm[2] == 4 && perm[3] == 0 && perm[4] == 2);
    CHECK(nao_partition_points(xyz, 5, 2, 1, off, perm, &nbat) == NAO_ERR_INVALID_ARG && nbat == 3);

    /* the natural spline through a quadratic's samples: c0 are the samples, M_0 = 0 at the ends */
    double y[8], coef[7 * 4];
    for (int k = 0; k < 8; k++) y[k] = 0.5 * k * k;
    CHECK(nao_radial_spline(y, 8, coef) == NAO_OK);
    for (int k = 0; k < 7; k++) CHECK(coef[4 * k] == y[k]);
    CHECK(coef[2] == 0.0);  /* c2 = M_0 / 2 = 0 */
    double end = coef[24] + coef[25] + coef[26] + coef[27];
    CHECK(fabs(end - y[7]) < 1e-12);
    CHECK(nao_radial_spline(y, 3, coef) == NAO_ERR_INVALID_ARG);
    printf("ok\n");
    return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_header_is_c11_and_host_entry_points_work_from_c():
    lib = nao.lib_path()
    if not lib.exists():
        pytest.skip("libnao.so not built")
    work = lib.parent / "ctest"
    work.mkdir(exist_ok=True)
    src, exe = work / "abi_check.c", work / "abi_check"
    src.write_text(PROGRAM)
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{ROOT / 'include'}", str(src), "-o", str(exe),
           f"-L{lib.parent}", "-lnao", f"-Wl,-rpath,{lib.parent}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
