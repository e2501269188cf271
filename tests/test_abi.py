"""The C-ABI library loads, exports every function declared in include/chns.h, and
rejects invalid leaf lists on the host before touching the GPU."""
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "chns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chns_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def chns():
    import paper_2009_06628_gb300 as chns
    if not os.path.exists(chns.LIB_PATH):
        from paper_2009_06628_gb300 import build
        build.build()
    chns.load()
    return chns


def test_every_declared_symbol_is_exported(chns):
    names = _declared_functions()
    assert len(names) >= 14
    lib = chns.load()
    for n in names:
        assert hasattr(lib, n), n
    bound = {s[0] for s in chns.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


def test_rejects_unsorted_leaves(chns):
    leaves = synth.uniform_leaves(2, 3)[::-1].copy()
    with pytest.raises(chns.ChnsError) as e:
        chns.Mesh(2, 3, leaves)
    assert e.value.name == "CHNS_ENOTSORTED"


@pytest.mark.parametrize("cut", ["gap", "overlap", "misaligned"])
def test_rejects_incomplete_leaves(chns, cut):
    leaves = synth.uniform_leaves(3, 2)
    if cut == "gap":
        leaves = leaves[np.arange(leaves.shape[0]) != 5].copy()
    elif cut == "overlap":
        extra = leaves.copy()
        extra[:, 3] = 1
        leaves = np.concatenate([leaves[:1], np.array([[0, 0, 0, 1]], dtype=np.int32), leaves[1:]])
    else:
        leaves = leaves.copy()
        leaves[3, 0] += 1
    with pytest.raises(chns.ChnsError) as e:
        chns.Mesh(3, 2, leaves)
    assert e.value.name in ("CHNS_ENOTCOMPLETE", "CHNS_ENOTSORTED")


@pytest.mark.parametrize("dim", [2, 3])
def test_rejects_unbalanced_octree(chns, dim):
    # one quadrant refined two levels beyond its neighbours, no balancing
    leaves = synth.refine_leaves(dim, 1, 3, lambda lo, hi, lev: np.all(hi <= 0.5 + 1e-12, axis=1))
    with pytest.raises(chns.ChnsError) as e:
        chns.Mesh(dim, 3, leaves)
    assert e.value.name == "CHNS_ENOTBALANCED"


def test_rejects_bad_arguments(chns):
    leaves = synth.uniform_leaves(2, 2)
    with pytest.raises(chns.ChnsError) as e:
        chns.Mesh(4, 2, leaves)
    assert e.value.name == "CHNS_EINVAL"
    with pytest.raises(chns.ChnsError) as e:
        chns.Mesh(2, 2, leaves, lo=1.0, hi=0.0)
    assert e.value.name == "CHNS_EINVAL"


def test_struct_layouts_match_the_header(chns, tmp_path):
    """The ctypes mirrors of chns_params, chns_solver_opts and chns_stats have the size and
    the field offsets that a C compiler gives the structs of include/chns.h (a field added
    on one side only, or reordered, fails here before any call passes a misread struct)."""
    import ctypes
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"chns_params": chns.Params, "chns_solver_opts": chns.SolverOpts, "chns_stats": chns.Stats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "chns.h"', "int main(void) {",
             '  printf("chns_leaf %zu\\n", sizeof(chns_leaf));']
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                text=True).stdout.splitlines())
    assert int(out["chns_leaf"]) == 16
    for cname, py in structs.items():
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_guess_option_needs_a_first_iterate(chns):
    """opts.guess = 1 starts Newton from U_out as passed, so the binding refuses the call
    without one (on the host, before the library is entered)."""
    import torch
    with pytest.raises(ValueError):
        chns.newton_step(None, None, chns.SolverOpts.make(guess=1), torch.zeros(4, 5, dtype=torch.float64))
