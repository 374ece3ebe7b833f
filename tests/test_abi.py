"""The C-ABI library builds, loads and exports every symbol that
include/dbg.h declares; host-only entry points behave (no GPU needed)."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2401_02756_gb300 import build, dbg, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dbg.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dbg_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert "dbg_insert_reads" in decl and "dbg_export_sorted" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(decl) == sorted(dbg.EXPORTED)


def test_library_is_built_for_sm103a_only():
    # every translation unit and the link take exactly one target, sm_103a
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any("arch" in f or "sm_" in f for f in build.FLAGS)


@pytest.mark.gpu
def test_kernels_report_sm103_at_run_time(lib):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    v = ctypes.c_int()
    assert lib.dbg_binary_version(ctypes.byref(v)) == dbg.OK
    assert v.value == 103


def test_strerror_and_status_names(lib):
    for code, name in dbg.STATUS_NAMES.items():
        assert lib.dbg_strerror(code)
    assert lib.dbg_strerror(99) == b"unknown status"


def test_pack_ascii_matches_generator_packing(lib):
    rng = np.random.default_rng(5)
    for n in (0, 1, 3, 4, 5, 31, 64, 1001):
        s = "".join(rng.choice(list("ACGT"), size=n))
        assert np.array_equal(dbg.pack_ascii(s), synth.pack_codes(synth.ascii_to_codes(s)))


def test_pack_ascii_phase_and_rejection(lib):
    out = dbg.pack_ascii("GT", phase=2)
    assert list(out) == [(2 << 4) | (3 << 6)]
    with pytest.raises(dbg.DbgError) as e:
        dbg.pack_ascii("ACGNA")
    assert e.value.code == dbg.ERR_INVALID_ARG and "at 3" in str(e.value)


def test_argument_errors_return_before_any_launch(lib):
    h = ctypes.c_void_p()
    assert lib.dbg_create(1, 10, ctypes.byref(h)) == dbg.ERR_INVALID_ARG
    assert lib.dbg_create(65, 10, ctypes.byref(h)) == dbg.ERR_INVALID_ARG
    assert lib.dbg_create(21, 0, ctypes.byref(h)) == dbg.ERR_INVALID_ARG
    assert lib.dbg_create(21, 10, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_insert_reads(None, None, None, 5, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_insert_reads_host(None, None, None, 5, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_build_reads(None, None, None, 5, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_build_reads_host(None, None, None, 0, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_binary_version(None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_insert_batch(None, 3, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_insert_batch(None, 0, None) == dbg.OK
    assert lib.dbg_get_status(None, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_stats(None, None, None, None) == dbg.ERR_INVALID_ARG
    n = ctypes.c_uint64()
    assert lib.dbg_export_sorted(None, None, None, 0, ctypes.byref(n), None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_probe_random_sectors(None, 1, 1, 0, 0, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_sketch_reads(1, None, None, 0, None, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_sketch_estimate(None) < 0
    assert lib.dbg_mlp_work_floats(0) == 0
    assert lib.dbg_mlp_work_floats(3) == 3 * (4 * dbg.MLP_HIDDEN + 2) + 1
    assert lib.dbg_mlp_features(None, 1025, 1, None, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_mlp_features(1, 1000, 1, 1, None) == dbg.ERR_INVALID_ARG  # stride < inputs
    assert lib.dbg_mlp_init(None, 0, None) == dbg.ERR_INVALID_ARG
    assert lib.dbg_mlp_forward(1, 1, 0, 1, 1, None) == dbg.ERR_INVALID_ARG  # empty batch
    assert lib.dbg_mlp_train_step(1, 1, 1, 1, 0, 1e-3, 1, 1, 4, 1, None, None) == \
        dbg.ERR_INVALID_ARG  # step 0
    assert lib.dbg_mlp_train_step(1, 1, 1, 1, 1, 0.0, 1, 1, 4, 1, None, None) == \
        dbg.ERR_INVALID_ARG  # lr 0
    lib.dbg_destroy(None)


def test_mlp_constants_match_the_reference_layout():
    from oracle import mlp
    assert (dbg.MLP_INPUTS, dbg.MLP_HIDDEN, dbg.MLP_PARAMS) == (mlp.IN, mlp.HID, mlp.N_PARAMS)
    txt = open(os.path.join(ROOT, "include", "dbg.h")).read()
    for name, v in (("INPUTS", mlp.IN), ("HIDDEN", mlp.HID), ("PARAMS", mlp.N_PARAMS)):
        assert re.search(rf"#define DBG_MLP_{name} {v}\b", txt)


def test_create_fails_loudly_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dbg.DbgError) as e:
        dbg.Graph(21, 1000)
    assert e.value.code in (dbg.ERR_CUDA, dbg.ERR_OOM)


def _c_struct_fields(name):
    txt = open(os.path.join(ROOT, "include", "dbg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = txt[txt.index(f"typedef struct {name} {{"):txt.index(f"}} {name};")]
    return re.findall(r"\b(?:int|uint64_t|uint32_t|dbg_handle)\s*\**\s*(\w+)\s*;", body)


def _c_struct_all_fields(name):
    txt = open(os.path.join(ROOT, "include", "dbg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    body = txt[txt.index(f"typedef struct {name} {{"):txt.index(f"}} {name};")]
    return re.findall(r"(\w+)\s*;", body)


def test_binding_structs_match_the_header(lib):
    assert [f for f, _ in dbg.Tuning._fields_] == _c_struct_fields("dbg_tuning")
    assert [f for f, _ in dbg.Info._fields_] == _c_struct_fields("dbg_info")
    assert list(dbg.Graph.TUNING_FIELDS) == _c_struct_fields("dbg_tuning")
    assert [f for f, _ in dbg.SketchItem._fields_] == _c_struct_all_fields("dbg_sketch_item")
    assert len(dbg.BatchItem._fields_) == len(_c_struct_all_fields("dbg_batch_item"))


def test_set_tuning_rejects_unknown_fields(lib):
    class Fake(dbg.Graph):
        def __init__(self):
            self._h = None
    with pytest.raises(ValueError):
        Fake().set_tuning(no_such_field=1)
