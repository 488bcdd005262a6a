"""The C-ABI library builds, loads and exports every symbol include/tl.h
declares; struct layouts agree between C and the binding; argument
validation runs on the host (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2110_12932_gb300 import build as tlbuild
from paper_2110_12932_gb300 import tl, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tl.h")


@pytest.fixture(scope="module")
def lib():
    tlbuild.build()
    return tl.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(tl_[a-z_]+)\s*\(", src))
    return sorted(n for n in names if n not in ("tl_track", "tl_config", "tl_stats"))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(tl.EXPORTS)


def _c_layout(struct, fields):
    """sizeof and offsetof from a C compile of the header."""
    body = "\n".join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    prog = f"""
#include <stdio.h>
#include <stddef.h>
#include "tl.h"
int main(void) {{ printf("%zu\\n", sizeof({struct})); {body} return 0; }}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("ctype,cname", [(tl.tl_config, "tl_config"), (tl.tl_stats, "tl_stats"),
                                         (tl.tl_track, "tl_track")])
def test_struct_layout_matches_header(ctype, cname):
    fields = [f for f, _ in ctype._fields_]
    lay = _c_layout(cname, fields)
    assert lay[0] == C.sizeof(ctype)
    for f, off in zip(fields, lay[1:]):
        assert getattr(ctype, f).offset == off, f


def _einval(lib, **over):
    cfg = workloads.workload("single_track_tiny")
    cfg.update(over)
    st, h = tl.tl_create_problem(cfg)
    assert not h.value
    return st


@pytest.mark.parametrize("over", [
    dict(r=0), dict(m=0), dict(pNXc=17), dict(pNZc=0), dict(NXc=0), dict(dt_coarse=0.0),
    dict(k0=-1.0), dict(rho=0.0), dict(radius=0.0), dict(tol=0.0), dict(max_iter=0),
    dict(tracks=[(0.0, 0.0, 1e-3, 1e-3, 0.8)]),          # diagonal track with the box source
    dict(tracks=[(0.0, 0.0, 1e-3, 0.0, 0.0)]),           # zero speed
    dict(coarse_source=2), dict(precision=7), dict(inner_tiles=3), dict(inner_tiles=-1),
    dict(precond=3), dict(precond=-1), dict(coupling_sweeps=2, coupling_tol=0.0),
    dict(picard_iters=51), dict(picard_iters=-1), dict(picard_iters=2, coupling_sweeps=2),
    dict(latent=-1.0), dict(latent=2.86e5, pc_sharpness=0.0), dict(latent=2.86e5, T_liquidus=1800.0),
    dict(h_conv=-1.0), dict(emissivity=1.5), dict(emissivity=-0.1), dict(h_conv=10.0, T_amb=0.0),
    dict(barrier_timeout=-1.0), dict(barrier_timeout=61.0), dict(h_conv=10.0, precond=1),
    dict(interface_coupling=2), dict(interface_coupling=1, coupling_sweeps=2, coupling_tol=1e-10), dict(autotune=2),
])
def test_invalid_config_is_rejected_on_host(lib, over):
    assert _einval(lib, **over) == tl.TL_EINVAL


def test_null_arguments(lib):
    assert lib.tl_create_problem(None, None) == tl.TL_EINVAL
    assert lib.tl_coarse_step(None, 0) == tl.TL_EINVAL
    assert lib.tl_fine_substeps(None, 1) == tl.TL_EINVAL
    assert lib.tl_restrict(None) == tl.TL_EINVAL
    assert lib.tl_node_count(None, 0) == 0
    lib.tl_destroy_problem(None)
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert tl.tl_status_string(s) != "unknown status"


def test_trace_mark_names_cover_the_kernel_marks():
    """Every phase marker the solve kernel records has a name in the binding."""
    with open(os.path.join(ROOT, "paper_2110_12932_gb300", "csrc", "tl_solve.cuh")) as f:
        src = f.read()
    body = src[src.index("enum TraceMark"):]
    body = body[:body.index("};")]
    values = {int(v) for v in re.findall(r"TR_[A-Z0-9_]+\s*=\s*(\d+)", body)}
    assert values and values == set(tl.TRACE_MARKS)
