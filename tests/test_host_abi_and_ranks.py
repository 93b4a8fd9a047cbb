"""CPU-only checks of the host side: the C-ABI library loads and exports every entry
point include/alm.h declares, the binding's struct layouts match the header, and the
multi-rank reduction of bench.py (replicas, max over ranks) works with gloo."""
import ctypes
import os
import re
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "alm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(alm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2505_15775_gb300 import build

    return build.build()  # nvcc cross-compiles for sm_103a without a GPU


def test_library_exports_every_declared_entry_point(lib_path):
    declared = _declared_functions()
    assert len(declared) >= 12
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(alm_\w+)", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)  # loads without a GPU
    for f in declared:
        assert hasattr(lib, f)


def test_binding_covers_the_header_and_struct_sizes(lib_path):
    from paper_2505_15775_gb300 import alm

    assert set(alm.EXPORTED) == set(_declared_functions())
    # struct layouts: compile a probe of sizeof/offsetof against the header with gcc
    probe = os.path.join(ROOT, "paper_2505_15775_gb300", "_build", "abi_probe")
    csrc = probe + ".c"
    os.makedirs(os.path.dirname(probe), exist_ok=True)
    with open(csrc, "w") as f:
        f.write('#include <stdio.h>\n#include <stddef.h>\n#include "alm.h"\nint main(void){'
                'printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(alm_problem), sizeof(alm_options), sizeof(alm_stats),'
                ' offsetof(alm_options, inner_precond), offsetof(alm_stats, lanczos_ms), sizeof(alm_batch_problem),'
                ' sizeof(alm_instance_stats), sizeof(alm_batch_stats));return 0;}\n')
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), csrc, "-o", probe], check=True)
    sizes = [int(x) for x in subprocess.run([probe], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(alm.alm_problem), ctypes.sizeof(alm.alm_options), ctypes.sizeof(alm.alm_stats),
                     alm.alm_options.inner_precond.offset, alm.alm_stats.lanczos_ms.offset,
                     ctypes.sizeof(alm.alm_batch_problem), ctypes.sizeof(alm.alm_instance_stats),
                     ctypes.sizeof(alm.alm_batch_stats)]
    o = alm.default_options()
    assert o.precision == alm.ALM_FP64 and o.r_max == 32 and o.inner_precond == 1


def test_library_calls_fail_cleanly_without_arguments(lib_path):
    from paper_2505_15775_gb300 import alm

    lib = alm.load()
    h = ctypes.c_void_p()
    assert lib.alm_create(ctypes.byref(h), None, None, None) == alm.ALM_ERR_INVALID_ARG
    assert not h.value
    assert b"NULL" in lib.alm_last_error(None)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_replica_time_is_max_over_ranks_gloo():
    code = (
        "import os, sys, torch.distributed as dist\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import bench\n"
        "dist.init_process_group('gloo')\n"
        "r = dist.get_rank()\n"
        "v = bench.max_over_ranks(1.5 + r, dist.get_world_size())\n"
        "assert v == 2.5, v\n"
        "dist.destroy_process_group()\n"
        "print('ok', r)\n"
    )
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
        assert o.startswith("ok")


def test_batch_and_network_reject_bad_input_on_the_host(lib_path):
    """Validation happens on the host before any CUDA call, so it is testable without a GPU."""
    import numpy as np

    from paper_2505_15775_gb300 import alm

    lib = alm.load()
    h = ctypes.c_void_p()
    row_off = np.array([0, 3, 5], np.int64)
    nnz_off = np.array([0, 2, 3], np.int64)
    ci = np.array([0, 1, 0], np.int32)
    cj = np.array([1, 2, 1], np.int32)
    cv = np.array([0.25, 0.25, 0.25])
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)

    def create(precision=alm.ALM_FP32, ci=ci, count=2):
        p = alm.alm_batch_problem(count=count, row_off=ptr(row_off), nnz_off=ptr(nnz_off), c_i=ptr(ci),
                                  c_j=ptr(cj), c_v=ptr(cv))
        o = alm.default_options(precision=precision)
        return lib.alm_batch_create(ctypes.byref(h), ctypes.byref(p), ctypes.byref(o), None)

    assert create(precision=alm.ALM_FP64) == alm.ALM_ERR_INVALID_ARG
    assert b"FP32" in lib.alm_batch_last_error(None)
    bad = ci.copy()
    bad[2] = 2  # (2, 1) in instance 1: not upper-triangle
    assert create(ci=bad) == alm.ALM_ERR_INVALID_ARG
    assert b"instance 1" in lib.alm_batch_last_error(None)
    assert create(count=0) == alm.ALM_ERR_INVALID_ARG
    assert not h.value
    assert lib.alm_gnn_create(ctypes.byref(h), 7, 0, 0, None) == alm.ALM_ERR_INVALID_ARG
    assert b"storage" in lib.alm_gnn_last_error(None)
    assert lib.alm_gnn_num_params() == 19713
