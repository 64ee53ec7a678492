"""CPU check of the tracing ranges: every C-ABI call opens an NVTX range named after it and closes
it on every return path, including argument errors.  A minimal NVTX v3 injection library (the
interface a profiler attaches through: NVTX_INJECTION64_PATH names a shared library exporting
InitializeInjectionNvtx2, which fills the core module's RangePushA / RangePop slots) is built
with gcc and logs the ranges; no GPU is needed because the calls fail their host checks."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Callback-table ids of the NVTX v3 injection interface: export table 1 = callbacks, module 1 =
# core, slot 9 = RangePushA, slot 11 = RangePop.
PROBE_C = textwrap.dedent(r"""
    #include <stddef.h>
    #include <stdint.h>
    #include <stdio.h>
    #include <stdlib.h>

    typedef void (*fnptr_t)(void);
    typedef fnptr_t **fntable_t;
    typedef struct {
        size_t struct_size;
        int (*get_module_table)(int module, fntable_t *table, unsigned int *size);
    } callbacks_t;
    typedef const void *(*get_export_t)(uint32_t id);

    static FILE *out;
    static int on_push(const char *name) { fprintf(out, "push %s\n", name); fflush(out); return 0; }
    static int on_pop(void) { fprintf(out, "pop\n"); fflush(out); return 0; }

    int InitializeInjectionNvtx2(get_export_t get)
    {
        const callbacks_t *cb = (const callbacks_t *)get(1);
        fntable_t t = NULL;
        unsigned int n = 0;
        const char *path = getenv("NVTX_PROBE_LOG");
        if (!cb || !path || !cb->get_module_table(1, &t, &n) || n < 12) return 0;
        out = fopen(path, "w");
        if (!out) return 0;
        *t[9] = (fnptr_t)on_push;
        *t[11] = (fnptr_t)on_pop;
        return 1;
    }
""")

CHILD = textwrap.dedent(r"""
    import ctypes, sys
    sys.path.insert(0, sys.argv[1])
    import numpy as np
    from paper_2512_12442_gb300 import _lib
    lib = _lib.load()
    X = np.zeros((4, 3)); y = np.zeros(4); ell = np.ones(3); h = ctypes.c_void_p()
    assert lib.gpr_model_create(X.ctypes.data, y.ctypes.data, 0, 0, ell.ctypes.data, 1.0, 1e-4, None,
                                ctypes.byref(h)) != 0
    assert lib.gpr_lcp_dense(None, None, 0.0, None, None, None, None) != 0
    assert lib.gpr_lcp_adaptive(None, None, 0.0, 3, None, None, None, None) != 0
""")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc for the injection probe")
def test_c_abi_calls_open_and_close_nvtx_ranges(tmp_path):
    from paper_2512_12442_gb300 import build
    build.build()
    src = tmp_path / "probe.c"
    src.write_text(PROBE_C)
    so = tmp_path / "libprobe.so"
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-o", str(so), str(src)], check=True)
    log = tmp_path / "ranges.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(so), NVTX_PROBE_LOG=str(log))
    subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, check=True, timeout=300)
    lines = log.read_text().split("\n")[:-1]
    assert lines == ["push gpr_model_create", "pop", "push gpr_lcp_dense", "pop", "push gpr_lcp_adaptive", "pop"]
