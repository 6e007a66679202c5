"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every declared symbol, its structs match the header byte for byte, and the
host-side logic (validation, workspace sizing) behaves."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "at.h")


@pytest.fixture(scope="module")
def L():
    from paper_2204_01133_gb300 import api, build
    build.build()
    return api.lib()


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^[a-z_ *]*?\b(at_[a-z_]+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("at_create", "at_set_problem", "at_set_delays", "at_step", "at_run", "at_read"):
        assert f in names


def test_library_exports_every_declared_symbol(L):
    from paper_2204_01133_gb300 import api
    names = declared_functions()
    assert set(names) == set(api.SYMBOLS)
    for f in names:
        assert hasattr(L, f), f
    out = subprocess.run(["nm", "-D", "--defined-only", api.LIB_PATH], capture_output=True, text=True).stdout
    for f in names:
        assert re.search(r"\bT %s$" % f, out, flags=re.M), f


def test_probe_library_exports_its_declared_symbols(L):
    from paper_2204_01133_gb300 import build
    src = open(os.path.join(ROOT, "include", "at_probe.h")).read()
    names = sorted(set(re.findall(r"^int (at_probe_[a-z0-9_]+)\s*\(", src, flags=re.M)))
    assert len(names) == 5
    out = subprocess.run(["nm", "-D", "--defined-only", build.PROBE], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (at_probe_[a-z0-9_]+)$", out, flags=re.M))
    assert exported == set(names)


def test_library_targets_sm103a_only(L):
    from paper_2204_01133_gb300 import api
    r = subprocess.run(["cuobjdump", "--list-elf", api.LIB_PATH], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in r.stdout
    assert "sm_90" not in r.stdout and "sm_100" not in r.stdout


def test_struct_layouts_match_header():
    from paper_2204_01133_gb300 import api
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "at.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(at_problem), offsetof(at_problem, n), offsetof(at_problem, prm),
         sizeof(at_delays), offsetof(at_delays, seed));
  printf("%zu %zu %zu %zu\n", offsetof(at_delays, instance), sizeof(at_stats), offsetof(at_stats, kernels_launched), offsetof(at_stats, stage_ms));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(prog)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(api.Problem), api.Problem.n.offset, api.Problem.prm.offset,
                    ctypes.sizeof(api.Delays), api.Delays.seed.offset, api.Delays.instance.offset,
                    ctypes.sizeof(api.Stats), api.Stats.kernels_launched.offset, api.Stats.stage_ms.offset]


def test_workspace_sizing_and_validation(L):
    from paper_2204_01133_gb300 import api
    from paper_2204_01133_gb300 import workloads as W
    pb, _ = W.advdiff()
    nb = api.workspace_bytes(pb)
    n, R, S, P, H = 2048, 3 + 2 + 1, 4, 32, 2
    field = 8 * n
    assert nb >= 3 * field + 8 * R * S * P * 2 * H + S * P * 2
    assert nb % 256 == 0
    # a larger delay model needs a larger ring
    assert api.workspace_bytes(dict(pb, k_max=6)) > nb
    # invalid descriptions are rejected with 0
    assert api.workspace_bytes(dict(pb, n=2049)) == 0
    assert api.workspace_bytes(dict(pb, n=0)) == 0            # empty domain
    assert api.workspace_bytes(dict(pb, pe_size=0)) == 0
    assert api.workspace_bytes(dict(pb, n=-64)) == 0
    assert api.workspace_bytes(dict(pb, pe_size=3)) == 0      # below 2 x halo width
    assert api.workspace_bytes(dict(pb, k_max=16)) == 0
    assert api.workspace_bytes(dict(pb, order=8)) == 0
    assert b"order" in L.at_last_error()
    assert api.workspace_bytes(dict(pb, n=2053 * 2, pe_size=2053)) == 0   # prime above 1024
    assert b"divisor" in L.at_last_error()
    assert api.workspace_bytes(dict(pb, n=263 * 3, pe_size=263)) > 0      # prime, one window


def test_calls_out_of_order_and_without_gpu(L):
    from paper_2204_01133_gb300 import api
    h = ctypes.c_void_p()
    rc = L.at_create(ctypes.byref(h), 0, None)
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        assert rc == api.AT_OK
        assert L.at_step(h, 1) == api.AT_ESTATE
        L.at_destroy(h)
    else:
        assert rc in (api.AT_ECUDA, api.AT_EINVAL)
        assert L.at_last_error()
    assert L.at_step(None, 1) == api.AT_EINVAL
    assert L.at_checkpoint_bytes(None) == 0
    assert L.at_save(None, None, 0, 0) == api.AT_EINVAL
    assert L.at_restore(None, None, 0, 0) == api.AT_EINVAL


def test_batch_table_and_validation(L):
    import ctypes
    from paper_2204_01133_gb300 import api, batch
    assert batch.table_bytes(0) == 0
    t1, t2 = batch.table_bytes(1), batch.table_bytes(4096)
    assert t1 > 0 and t2 > t1 and t2 % 256 == 0
    assert batch.table_bytes(16, 1 << 20) > batch.table_bytes(16, 16) + 8 * ((1 << 20) - 16) - 512
    h = ctypes.c_void_p()
    batch._lib()
    # a misaligned or too small table is refused before any CUDA call
    assert L.at_batch_create(ctypes.byref(h), 0, None, 16, 64, ctypes.c_void_p(256 + 8), 1 << 20) == api.AT_EINVAL
    assert L.at_batch_create(ctypes.byref(h), 0, None, 16, 64, ctypes.c_void_p(256), 16) == api.AT_ENOMEM
    assert L.at_batch_create(ctypes.byref(h), 0, None, 0, 64, ctypes.c_void_p(256), 1 << 20) == api.AT_EINVAL


def test_enum_values_match_the_binding():
    """Every AT_* enumerator of include/at.h has the value the Python binding
    passes for it (no GPU needed)."""
    import re
    from paper_2204_01133_gb300 import api, batch
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(AT_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}

    def binding(name):  # the binding's constant for one enumerator, or None
        short = name[3:]
        if short.startswith("BATCH_"):
            return getattr(batch, short[6:], None)
        for table in (api.PDE, api.RK, api.MODE, api.DIST):
            if short.lower() in table:
                return table[short.lower()]
        return getattr(api, short, getattr(api, name, None))

    found = {name: binding(name) for name in values}
    for name, value in values.items():
        assert found[name] == value, (name, value, found[name])
    for name in ("AT_PATH_FUSED", "AT_OPT_WITHHOLD_PE", "AT_ETIMEOUT", "AT_READ_STATS", "AT_BATCH_FLAT",
                 "AT_RNS_CHAIN", "AT_GEOMETRIC"):
        assert name in values
    assert len(values) >= 36


def test_noalloc_scratch_size_matches_the_binding():
    """AT_NOALLOC_SCRATCH_BYTES of include/at.h (a #define, not an
    enumerator) equals the binding's NOALLOC_SCRATCH_BYTES."""
    import re
    from paper_2204_01133_gb300 import api
    m = re.search(r"#define\s+AT_NOALLOC_SCRATCH_BYTES\s+\(\(size_t\)(\d+)\s*<<\s*(\d+)\)", open(HEADER).read())
    assert m, "AT_NOALLOC_SCRATCH_BYTES is not of the form ((size_t)A << B)"
    assert int(m.group(1)) << int(m.group(2)) == api.NOALLOC_SCRATCH_BYTES


def test_exp_table_is_what_its_generator_writes():
    """csrc/exp_table.h is generated from the definitions 2^(j/256) and
    ln 2 / 256 in high-precision decimal arithmetic; the committed file must
    be exactly the generator's output, and its table must hold 2^(j/256)
    rounded to double."""
    import math
    import subprocess
    import sys
    csrc = os.path.join(ROOT, "paper_2204_01133_gb300", "csrc")
    out = subprocess.run([sys.executable, os.path.join(csrc, "gen_exp_table.py")], capture_output=True, text=True,
                         check=True).stdout
    with open(os.path.join(csrc, "exp_table.h")) as f:
        assert f.read().strip() == out.strip()
    vals = [float.fromhex(t) for line in out.splitlines() if line.startswith("    0x")
            for t in line.strip().rstrip(",").split(", ")]
    assert len(vals) == 256
    assert all(abs(v - 2.0 ** (j / 256)) <= math.ulp(v) for j, v in enumerate(vals))
