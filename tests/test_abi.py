"""The C ABI boundary on the CPU: the library builds for sm_103a, loads, and exports every
entry point that include/nd.h declares; the binding wraps each of them. No kernel runs."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^ND_API\s+[\w\s\*]*?\b(nd_\w+)\(", txt, flags=re.M))
    return names


def test_header_declares_the_hot_path_calls():
    names = declared_symbols()
    for n in ["nd_load_csr", "nd_orient", "nd_count", "nd_decompose", "nd_ctx_create", "nd_last_error",
              "nd_rounds", "nd_round_times", "nd_batch_run", "nd_server_create", "nd_submit", "nd_poll"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2111_10980_gb300 as nd
    from paper_2111_10980_gb300 import build

    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nd_\w+)$", out, flags=re.M))
    missing = declared_symbols() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    # nothing but the declared API is exported
    extra = {s for s in exported if s.startswith("nd_")} - declared_symbols()
    assert not extra, f"exported but not declared: {sorted(extra)}"
    L = nd.lib()
    for name in declared_symbols():
        assert hasattr(L, name)
    assert set(nd.API) == declared_symbols()


def test_built_for_sm_103a_only():
    """The build compiles every translation unit and links with exactly one target,
    -gencode arch=compute_103a,code=sm_103a (a GB300 cubin and no PTX, so nothing can be
    JIT-compiled for another architecture), with line info for the profiler."""
    from paper_2111_10980_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    cmds = build.commands()
    assert cmds and all(c[c.index("-gencode") + 1] == "arch=compute_103a,code=sm_103a" for c in cmds)
    assert all(c.count("-gencode") == 1 for c in cmds)
    assert all("-lineinfo" in c for c in cmds if "-c" in c)
    assert {os.path.basename(c[c.index("-c") + 1]) for c in cmds if "-c" in c} == \
        {os.path.basename(p) for p in build.sources()}


def test_error_path_without_gpu():
    """Argument errors are reported through nd_last_error without touching a device."""
    import ctypes

    import paper_2111_10980_gb300 as nd

    L = nd.lib()
    rc = L.nd_ctx_create(0, None, 0, None)
    assert rc == nd.ND_EINVAL
    assert "NULL" in nd.nd_last_error()
    assert L.nd_graph_free(None) == nd.ND_OK
    assert L.nd_orient(None, 0) == nd.ND_EINVAL
    assert L.nd_decompose(None, 2, 3, 0, None, None, 0, None) == nd.ND_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's size and field offsets (compiled as C)."""
    import ctypes

    import paper_2111_10980_gb300 as nd

    structs = {"nd_stats": nd.nd_stats, "nd_request": nd.nd_request, "nd_batch_stats": nd.nd_batch_stats,
               "nd_server_cfg": nd.nd_server_cfg, "nd_result": nd.nd_result}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "nd.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
