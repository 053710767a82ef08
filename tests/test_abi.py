"""The C-ABI library loads and exports every entry point include/vpmc.h
declares (no GPU needed: no compute call is made)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vpmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vpmc_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2307_01416_gb300 import build_ext, vpmc
    build_ext.build()
    L = vpmc.lib()
    names = _declared()
    assert "vpmc_run_spots" in names and "vpmc_influence_matrix" in names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", vpmc.LIB_PATH], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(r"\bT %s\b" % n, out), n
    assert sorted(vpmc.EXPORTED) == sorted(n for n in names)


def test_default_opts_without_gpu():
    from paper_2307_01416_gb300 import vpmc
    import ctypes as C
    o = vpmc.vpmc_opts()
    vpmc.lib().vpmc_default_opts(C.byref(o))
    assert (o.seed, o.mcs, o.straggling, o.nuclear, o.frac_bits, o.aggregate) == (1234, 1, 1, 1, 24, -1)


def test_binding_refuses_without_cuda(monkeypatch):
    import torch
    from paper_2307_01416_gb300 import vpmc, workloads as W
    if torch.cuda.is_available():
        pytest.skip("CUDA present")
    pb, _ = W.pencil_beam_water(n_hist=10)
    with pytest.raises(RuntimeError):
        vpmc.Engine(pb)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets of
    the C struct of the same name in include/vpmc.h (compiled with gcc)."""
    import ctypes as C
    from paper_2307_01416_gb300 import vpmc
    structs = {n: getattr(vpmc, n) for n in dir(vpmc)
               if n.startswith("vpmc_") and isinstance(getattr(vpmc, n), type)
               and issubclass(getattr(vpmc, n), C.Structure)}
    assert {"vpmc_beam", "vpmc_spot", "vpmc_opts", "vpmc_csr", "vpmc_opt_params"} <= set(structs)
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "vpmc.h"', "int main(void) {"]
    for n, cls in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (n, n))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (n, f[0], n, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        parts = line.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for n, cls in structs.items():
        assert got[(n, "size")] == C.sizeof(cls), n
        for f in cls._fields_:
            assert got[(n, f[0])] == getattr(cls, f[0]).offset, (n, f[0])
