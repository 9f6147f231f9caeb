"""The C-ABI library loads on the CPU host and exports every symbol the header declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eig_update.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(eig_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1706_00773_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("eig_update_init", "eig_update_rank_k", "eig_update_batch", "eig_update_query",
                 "eig_update_destroy", "eig_make_rank2"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_names_match_header(built_lib):
    import paper_1706_00773_gb300 as eu

    for name in _declared():
        assert callable(getattr(eu, name)), name
    assert eu.eig_version().startswith("eigupdate-gb300")


def test_constants_match_header():
    import paper_1706_00773_gb300 as eu

    txt = open(HEADER).read()
    for name in ("EIG_OK", "EIG_EINVAL", "EIG_ENOMEM", "EIG_ENOTCONV", "EIG_ETIMEOUT", "EIG_ECUDA",
                 "EIG_ENOTSUP", "EIG_EBUSY", "EIG_MAX_K", "EIG_Q_STATUS", "EIG_Q_REPORT",
                 "EIG_Q_LAST_STATUS", "EIG_Q_COUNT", "EIG_Q_WORKSPACE", "EIG_Q_METRICS"):
        m = re.search(r"#define %s \(?(-?\d+)\)?" % name, txt)
        assert m, name
        assert getattr(eu, name) == int(m.group(1)), name
    for name in ("EIG_FP64", "EIG_MIXED", "EIG_VALUES", "EIG_VECTORS", "EIG_REPORT", "EIG_ASYNC"):
        m = re.search(r"#define %s (\d+)u" % name, txt)
        assert m and getattr(eu, name) == int(m.group(1)), name


def test_init_without_gpu_fails_cleanly(built_lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    import paper_1706_00773_gb300 as eu

    with pytest.raises(eu.EigError) as ei:
        eu.eig_update_init(0)
    assert ei.value.code == eu.EIG_ECUDA
    # the failing runtime call is recorded for the thread and carried by the error
    code, msg = eu.eig_last_cuda_error()
    assert code != 0 and "cudaGetDeviceCount" in msg, (code, msg)
    assert "cudaGetDeviceCount" in ei.value.detail


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the header's size and field
    offsets (a C program compiled against the header prints them)."""
    import paper_1706_00773_gb300 as eu

    structs = {name: getattr(eu, name) for name in ("eig_init_params", "eig_problem", "eig_report", "eig_metrics",
                                                     "eig_count_args", "eig_server_params", "eig_request_info")}
    renames = {"lambda_": "lambda"}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "eig_update.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            cf = renames.get(f, f)
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, cf))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), "-o", str(exe), str(src)])
    got = {}
    for ln in subprocess.check_output([str(exe)], text=True).splitlines():
        a, b, c = ln.split()
        got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
