"""The C ABI from plain C: a C99 program that includes include/fpsa.h (compiled with
-pedantic -Werror), takes the address of every entry point, links against libfpsa.so and
calls the host-only ones with no GPU: fpsa_strerror for every status code and
fpsa_tables for S4, whose Gauss-Legendre weights sum to 2 and whose D M is the identity
(Eqs. phi-mom, treq); argument checks that precede any CUDA call return FPSA_EINVAL."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_LIB = "/usr/local/cuda/lib64"

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "fpsa.h"

typedef void (*entry_fn)(void);

int main(void) {
    entry_fn entry[] = {(entry_fn)fpsa_create, (entry_fn)fpsa_set_xs, (entry_fn)fpsa_set_incident, (entry_fn)fpsa_solve,
                     (entry_fn)fpsa_solve_batch, (entry_fn)fpsa_adjoint, (entry_fn)fpsa_destroy, (entry_fn)fpsa_strerror,
                     (entry_fn)fpsa_last_error, (entry_fn)fpsa_profile_enable, (entry_fn)fpsa_profile_read,
                     (entry_fn)fpsa_get_tuning, (entry_fn)fpsa_set_tuning, (entry_fn)fpsa_autotune, (entry_fn)fpsa_tables,
                     (entry_fn)fpsa_set_limits, (entry_fn)fpsa_sweep_noalloc};
    int codes[] = {FPSA_OK, FPSA_EINVAL, FPSA_ENOMEM, FPSA_ENONFINITE, FPSA_ENOTCONV, FPSA_EPIVOT,
                   FPSA_ETIMEOUT, FPSA_ECUDA, FPSA_ENOTSUP, FPSA_ESTATE};
    double mu[4], w[4], D[16], M[16], A[16];
    size_t i;
    int l, k, n;
    for (i = 0; i < sizeof entry / sizeof entry[0]; ++i)
        if (!entry[i]) return 10;
    for (i = 0; i < sizeof codes / sizeof codes[0]; ++i) {
        const char *s = fpsa_strerror(codes[i]);
        if (!s || !strlen(s)) return 11;
    }
    if (fpsa_tables(4, 4, FPSA_LAPLACIAN_MPD, mu, w, D, M, A) != FPSA_OK) return 12;
    if (fabs(w[0] + w[1] + w[2] + w[3] - 2.0) > 1e-14 || !(mu[0] < mu[1] && mu[2] < mu[3])) return 13;
    for (l = 0; l < 4; ++l)
        for (k = 0; k < 4; ++k) {
            double s = 0.0;
            for (n = 0; n < 4; ++n) s += D[l * 4 + n] * M[n * 4 + k];
            if (fabs(s - (l == k)) > 1e-13) return 14;
        }
    if (fpsa_tables(3, 1, FPSA_LAPLACIAN_MPD, mu, w, NULL, NULL, NULL) != FPSA_EINVAL) return 15;
    if (fpsa_create(NULL, NULL) != FPSA_EINVAL) return 16;
    printf("c caller ok\n");
    return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_1907_13013_gb300 import binding
    return binding.load()


def test_c_program_uses_the_library(tmp_path, lib):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc missing")
    src = tmp_path / "caller.c"
    src.write_text(PROGRAM)
    exe = str(tmp_path / "caller")
    libdir = os.path.join(ROOT, "paper_1907_13013_gb300")
    cmd = [gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
           str(src), "-o", exe, "-L" + libdir, "-lfpsa", "-Wl,-rpath," + libdir, "-lm"]
    if os.path.isdir(CUDA_LIB):
        cmd += ["-Wl,-rpath-link," + CUDA_LIB]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ)
    if os.path.isdir(CUDA_LIB):
        env["LD_LIBRARY_PATH"] = CUDA_LIB + os.pathsep + env.get("LD_LIBRARY_PATH", "")
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120, env=env)
    assert run.returncode == 0 and "c caller ok" in run.stdout, (run.returncode, run.stdout, run.stderr)
