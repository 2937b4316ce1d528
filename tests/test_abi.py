"""The C-ABI library builds, loads and exports every function include/trees.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1608_00571_b300 as trees
from paper_1608_00571_b300 import build as tbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "trees.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(trees_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    return tbuild.build()


def test_header_declares_functions():
    names = header_functions()
    assert "trees_run" in names and "trees_create" in names and len(names) >= 15


def test_library_exports_every_declared_function(libpath):
    out = subprocess.check_output(["nm", "-D", "--defined-only", libpath], text=True)
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_header(libpath):
    assert set(header_functions()) == set(trees.exported_symbols())
    L = trees.lib()
    for n in header_functions():
        assert hasattr(L, n)


def test_struct_sizes_match_header(libpath, tmp_path):
    # compile a tiny C program against the header and compare sizeof with ctypes
    c = tmp_path / "sz.c"
    c.write_text('#include <stdio.h>\n#include "trees.h"\nint main(){printf("%zu %zu %zu %zu\\n",'
                 'sizeof(trees_config_t),sizeof(trees_job_t),sizeof(trees_stats_t),sizeof(trees_epoch_t));}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    sizes = [int(x) for x in subprocess.check_output([str(exe)], text=True).split()]
    assert sizes == [ctypes.sizeof(trees.trees_config_t), ctypes.sizeof(trees.trees_job_t),
                     ctypes.sizeof(trees.trees_stats_t), ctypes.sizeof(trees.trees_epoch_t)]


def test_default_config_without_gpu(libpath):
    cfg = trees.trees_default_config()
    assert cfg.block_size == 512 and cfg.scheduler == trees.TREES_SCHED_PERSISTENT
    assert cfg.inject_stall_epoch == -1
    assert trees.trees_bytes_for(1000, cfg) > 1000 * 24
    assert trees.trees_bytes_for(0, cfg) == 0


def test_autotune_cache_hit_needs_no_gpu(libpath, tmp_path):
    # a cached key is answered from the JSON file before any device work
    cache = tmp_path / "tune.json"
    cache.write_text('{\n  "fib:n=34": {"block_size": 256, "tasks_per_thread": 4, "scheduler": 1, "ms": 0.5}\n}\n')
    best, ms, cands = trees.trees_autotune(trees.make_job(trees.TREES_PROG_FIB, n=34), 1 << 20,
                                           cache_path=str(cache), key="fib:n=34")
    assert (best.block_size, best.tasks_per_thread, best.scheduler) == (256, 4, 1)
    assert ms == 0.5 and cands == []
