"""The C ABI library: loads without a GPU, exports what include/bf.h declares,
rejects bad arguments, and its host-side double-precision decision tables
agree exactly with the FP64 oracle's per-pixel decisions."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth
from paper_2311_00482_gb300 import build as bfbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bf.h")


@pytest.fixture(scope="module")
def lib():
    bfbuild.build()
    return bf.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"BF_API\s+[\w\s\*]+?\b(bf_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for must in ("bf_create", "bf_submit", "bf_poll", "bf_destroy", "bf_beamform",
                 "bf_batch_create", "bf_last_error"):
        assert must in names
    assert set(names) == set(bf.EXPORTED)


def header_constants():
    """BF_* enumerators of include/bf.h with their values (plain integers and
    n << k forms)."""
    text = open(HEADER).read()
    consts = {}
    for body in re.findall(r"enum\s*\{([^}]*)\}", text):
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        for name, expr in re.findall(r"\b(BF_\w+)\s*=\s*([-\w\s<|]+?)\s*(?:,|$)", body):
            consts[name] = int(eval(expr, {}, dict(consts)))
    return consts


def test_binding_constants_match_the_header():
    consts = header_constants()
    assert {"BF_DAS", "BF_OUT_LOGDB", "BF_IQDAS", "BF_FK_STOLT", "BF_DEST_ONE_BUFFER",
            "BF_EINVAL"} <= set(consts)
    for name, value in consts.items():
        assert getattr(bf, name) == value, name


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert lib.bf_version() >= 100


def test_bad_arguments_are_rejected_without_a_gpu(lib):
    grid = (16, 16, -1e-3, 1e-3, 5e-3, 6e-3)
    cases = [
        dict(n_elements=0), dict(f_number=0.0), dict(f_number=-1.0), dict(pitch_m=0.0),
        dict(grid=(0, 16, -1e-3, 1e-3, 5e-3, 6e-3)), dict(grid=(16, 16, 1e-3, -1e-3, 5e-3, 6e-3)),
        dict(grid=(16, 16, -1e-3, 1e-3, -5e-3, 6e-3)), dict(grid=(16, 16, -1e-3, 1e-3, 6e-3, 5e-3)),
        dict(fs_hz=0.0), dict(c_mps=float("nan")), dict(grid=(40000, 16, 0, 1e-3, 5e-3, 6e-3)),
        dict(x_elem_m=[0.0, 0.0, 1e-3]),
    ]
    for bad in cases:
        args = dict(n_elements=3, pitch_m=3e-4, f_number=1.5, grid=grid, fs_hz=20e6, f0_hz=5e6,
                    c_mps=1540.0)
        args.update(bad)
        with pytest.raises(bf.BFError) as ei:
            bf.bf_create(**args)
        assert ei.value.code == bf.BF_EINVAL, bad
        assert bf.bf_last_error()


def test_pdas_order_needs_a_handle(lib):
    with pytest.raises(bf.BFError) as ei:
        bf.bf_set_pdas_order(None, 2.0)
    assert ei.value.code == bf.BF_EINVAL


def _compare_tables_with_oracle(acq, angles_rad, ns, x_elem=None):
    grid = (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)
    xe = acq.x_elements() if x_elem is None else np.asarray(x_elem)
    valid, cnt = bf.bf_host_tables(len(xe), acq.pitch_m, acq.f_number, grid, acq.fs_hz, acq.f0_hz,
                                   acq.c_mps, ns, angles_rad, x_elem_m=xe if x_elem is not None else None)
    empty = valid[..., 0] > valid[..., 1]
    assert not np.any(empty), "an empty row range is encoded as (-1, -1), never first > last"
    none = valid[..., 1] < 0
    assert np.all(valid[none] == -1)
    rf = np.zeros((len(angles_rad), len(xe), ns), np.int16)
    iz = np.arange(acq.nz)
    for ix in range(acq.nx):
        lo, hi = valid[:, ix, :, 0], valid[:, ix, :, 1]  # [A][N]
        for z in range(acq.nz):
            _, act, rec = oracle.delayed_samples(rf, xe, angles_rad, grid, ix, z, acq.fs_hz,
                                                 acq.c_mps, acq.f_number)
            counts = act & rec
            lib_counts = (lo <= z) & (z <= hi)
            assert np.array_equal(counts, lib_counts), (ix, z)
            assert cnt[ix, z] == act[0].sum()
    del iz


def test_host_tables_match_oracle_decisions_record_bound(lib):
    # 1024 samples: the deepest pixels of the 40 mm field fall beyond the record for
    # far elements, so the upper record bound is exercised; three compounded angles
    acq = synth.SPECKLE_POINTS_128.with_(nx=13, nz=29)
    _compare_tables_with_oracle(acq, np.deg2rad([-10.0, 0.0, 7.0]), 1024)


def test_host_tables_match_oracle_decisions_short_record_and_edges(lib):
    acq = synth.Acquisition(n_elements=24, nx=9, nz=41, z0_m=0.0, z1_m=20e-3, x0_m=-5e-3,
                            x1_m=5e-3, f_number=0.8)
    _compare_tables_with_oracle(acq, np.deg2rad([-25.0, 3.0]), 200)


def test_host_tables_inclusive_aperture_tie(lib, golden_dir):
    import json
    tie = json.load(open(os.path.join(golden_dir, "aperture_counts.json")))["edge_tie"]
    x, z = tie["pixel_m"]
    valid, cnt = bf.bf_host_tables(3, 1.0, tie["f_number"], (1, 1, x, x, z, z), 20e6, 5e6, 1540.0,
                                   256, [0.0], x_elem_m=tie["x_elem_m"])
    got = [(valid[0, 0, i, 0] <= 0 <= valid[0, 0, i, 1]) for i in range(3)]
    assert got == tie["active"] and cnt[0, 0] == 2
