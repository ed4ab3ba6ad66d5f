"""C-ABI checks that need no GPU: the library builds, loads, exports every function that
include/*.h declares, its structs have the sizes the binding assumes, and argument
validation that happens before any CUDA call returns DWF_EINVAL."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1101_0423_gb300 import build, dwf
    build.build()
    return dwf.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dwf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def declared_prototypes():
    """{name: (return type, [parameter declarations])} of every function include/*.h declares."""
    protos = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*((?:const\s+)?[A-Za-z_]\w*\s*\**)\s*(dwf_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M):
            params = [p.strip() for p in m.group(3).split(",") if p.strip() and p.strip() != "void"]
            protos[m.group(2)] = (m.group(1).strip(), params)
    return protos


def _ctype_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or t.__name__.startswith("LP_"):
        return "ptr"
    return {ctypes.c_int: "int", ctypes.c_uint: "unsigned", ctypes.c_double: "double",
            ctypes.c_uint64: "uint64_t"}[t]


def _c_kind(decl):
    if "*" in decl or "[" in decl:
        return "ptr"
    words = decl.replace("const", " ").split()
    base = words[0] if len(words) > 1 else words[0]
    return {"dwf_status": "int", "int": "int", "unsigned": "unsigned", "double": "double",
            "uint64_t": "uint64_t", "void": "void"}[base]


def test_binding_prototypes_match_the_header(lib):
    """Every ctypes prototype of the binding has the header's parameter count and kinds
    (pointer / int / unsigned / double / uint64_t) and its return kind."""
    protos = declared_prototypes()
    assert "dwf_apply_eo_dev_static" in protos
    assert set(protos) == set(declared_functions())
    for name, (ret, params) in protos.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, f"{name}: no ctypes prototype"
        got = [_ctype_kind(t) for t in f.argtypes]
        want = [_c_kind(p) for p in params]
        assert got == want, f"{name}: binding {got} vs header {want}"
        assert _ctype_kind(f.restype) == _c_kind(ret), f"{name}: return kind"


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["dwf_create", "dwf_destroy", "dwf_load_gauge", "dwf_apply_eo", "dwf_solve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    so = os.path.join(ROOT, "paper_1101_0423_gb300", "libdwf_gb300.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        assert hasattr(lib, n)


def test_struct_layouts_match_header(tmp_path):
    from paper_1101_0423_gb300 import dwf
    src = tmp_path / "sz.c"
    src.write_text('#include "dwf.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(dwf_solve_params), sizeof(dwf_solve_stats),'
                   ' offsetof(dwf_solve_stats, kernel_launches), offsetof(dwf_solve_params, profile));'
                   'printf("%zu %zu\\n", offsetof(dwf_solve_params, schur_target_pct),'
                   ' offsetof(dwf_solve_params, use_x0));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sp, ss, off_kl, off_prof, off_pct, off_x0 = map(int, subprocess.check_output([str(exe)]).split())
    assert sp == ctypes.sizeof(dwf.SolveParams)
    assert ss == ctypes.sizeof(dwf.SolveStats)
    assert off_kl == dwf.SolveStats.kernel_launches.offset
    assert off_prof == dwf.SolveParams.profile.offset
    assert off_pct == dwf.SolveParams.schur_target_pct.offset
    assert off_x0 == dwf.SolveParams.use_x0.offset


def test_defaults_and_status_strings(lib):
    from paper_1101_0423_gb300 import dwf
    p = dwf.dwf_solve_params_default()
    assert p.tol == 1e-10 and p.inner_prec == dwf.PREC_F32 and p.schur_parity == 1
    assert p.schur_target_pct == 50 and p.use_x0 == 0
    assert lib.dwf_status_string(dwf.DWF_ENOCONV) == b"DWF_ENOCONV"


@pytest.mark.parametrize("dims,ns,m0,omega_ok", [((3, 4, 4, 4), 4, 1.8, True), ((4, 4, 4, 4), 0, 1.8, True),
                                                  ((4, 4, 4, 4), 4, 2.5, True), ((4, 4, 4, 4), 4, 1.8, False)])
def test_create_rejects_invalid_arguments_before_touching_cuda(lib, dims, ns, m0, omega_ok):
    from paper_1101_0423_gb300 import dwf
    n = max(ns, 1)
    om = np.ones(n) if omega_ok else -np.ones(n)
    with pytest.raises(dwf.DwfError) as e:
        dwf.dwf_create(dims, ns, m0, 0.05, om, np.zeros(n))
    assert e.value.status == dwf.DWF_EINVAL


@pytest.mark.parametrize("ns", [1, 2, 5, 8, 16, 24, 64])
@pytest.mark.parametrize("kind", ["shamir", "borici", "cosine", "random"])
@pytest.mark.parametrize("mq", [0.0, 0.02, 0.7])
def test_create_builds_the_m5_recurrence_for_any_valid_weights(lib, ns, kind, mq):
    """dwf_create derives M5 and M5^T of Eq. 8 twice -- dense, from the cyclic bidiagonal
    structure, and as the recurrence tables of the FP64 hop epilogue -- and refuses the
    context (DWF_EINVAL) if the two disagree anywhere; this happens before any CUDA call.
    So a valid configuration may only fail later, at CUDA (no GPU here), never with EINVAL."""
    from paper_1101_0423_gb300 import dwf, inputs
    if kind == "random":
        rng = np.random.default_rng(ns)
        om, sg = rng.uniform(0.3, 1.7, ns), rng.uniform(-0.5, 1.2, ns)
    else:
        om, sg = inputs.weights(kind, ns)
    try:
        h = dwf.dwf_create((4, 4, 4, 4), ns, 1.8, mq, om, sg)
    except dwf.DwfError as e:
        assert e.status != dwf.DWF_EINVAL, "recurrence tables disagree with the dense M5"
    else:
        dwf.dwf_destroy(h)


def test_debug_wait_hook_rejects_a_null_context(lib):
    from paper_1101_0423_gb300 import dwf
    assert lib.dwf_debug_set_wait(None, 0, 1) == dwf.DWF_EINVAL


def test_server_struct_layouts_match_header(tmp_path):
    from paper_1101_0423_gb300 import dwf
    src = tmp_path / "sz2.c"
    src.write_text('#include "dwf.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(dwf_server_params),'
                   ' sizeof(dwf_request), sizeof(dwf_result), sizeof(dwf_server_stats),'
                   ' offsetof(dwf_server_stats, cancelled), offsetof(dwf_request, params));return 0;}\n')
    exe = tmp_path / "sz2"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sp, rq, rs, ss, off_c, off_p = map(int, subprocess.check_output([str(exe)]).split())
    assert sp == ctypes.sizeof(dwf.ServerParams)
    assert rq == ctypes.sizeof(dwf.Request) and off_p == dwf.Request.params.offset
    assert rs == ctypes.sizeof(dwf.Result)
    assert ss == ctypes.sizeof(dwf.ServerStats) and off_c == dwf.ServerStats.cancelled.offset


def test_partition_struct_layouts_match_header(tmp_path):
    """dwf_partition and dwf_part_comm (the domain decomposition's C structs) as the binding
    lays them out."""
    from paper_1101_0423_gb300 import dwf
    src = tmp_path / "sz3.c"
    src.write_text('#include "dwf.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(dwf_partition),'
                   ' offsetof(dwf_partition, coord), sizeof(dwf_part_comm),'
                   ' offsetof(dwf_part_comm, exchange), offsetof(dwf_part_comm, allreduce));return 0;}\n')
    exe = tmp_path / "sz3"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sp, off_coord, sc, off_ex, off_ar = map(int, subprocess.check_output([str(exe)]).split())
    assert sp == ctypes.sizeof(dwf.Partition) and off_coord == dwf.Partition.coord.offset
    assert sc == ctypes.sizeof(dwf.PartComm)
    assert off_ex == dwf.PartComm.exchange.offset and off_ar == dwf.PartComm.allreduce.offset
