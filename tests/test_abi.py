"""The C-ABI library builds, loads and exports every symbol include/srdr.h
declares; its host-side Philox4x64-10 matches numpy's bit generator and the
oracle's (no GPU needed for these calls)."""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_08932_gb300 import build as B
from paper_2103_08932_gb300 import srdr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return srdr.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "srdr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srdr_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(L):
    names = _declared()
    assert len(names) >= 16
    for name in names:
        assert hasattr(L, name), name
    assert sorted(srdr.EXPORTS) == names


def test_library_philox_matches_numpy_and_oracle(L):
    rng = np.random.default_rng(0)
    for _ in range(200):
        seed = int(rng.integers(0, 2**63))
        step = int(rng.integers(1, 2**40))
        mine = srdr.srdr_philox4x64_10([step, 0, 0, 0], [seed, 0])
        bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                              counter=np.array([step - 1, 0, 0, 0], dtype=np.uint64))
        assert list(mine) == list(bg.random_raw(4))
    for seed in (0, 1, 2, 3):
        for step in range(0, 20000, 7):
            assert srdr.srdr_random_phi(seed, step) == O.phi(seed, step)


def test_invalid_description_is_rejected_without_gpu(L):
    d = srdr.srdr_body_desc()
    d.dim = 4
    with pytest.raises(srdr.SrdrError) as e:
        srdr.srdr_body_create(d)
    assert e.value.status == srdr.SRDR_ERR_INVALID
    assert "dim" in srdr.last_error()


def test_entry_points_reject_null_handles_without_gpu(L):
    """Body, batch and control entry points (and the failure-path hook) check
    their handles on the host before any device call."""
    calls = [
        lambda: L.srdr_body_sweep_sync(None, srdr.SRDR_SWEEP_CELLS),
        lambda: L.srdr_body_sweep_lanes(None, 16),
        lambda: L.srdr_body_debug_stall_sweep(None),
        lambda: L.srdr_body_tune(None, 1, 1),
        lambda: L.srdr_body_pass_mapping(None, srdr.SRDR_PASS_SELL, 0, 0, 0),
        lambda: L.srdr_body_step(None, 1),
        lambda: L.srdr_body_relax(None, 1e-8, 10, None, None),
        lambda: L.srdr_body_read_displacement(None, None, 0),
        lambda: L.srdr_body_read_velocity(None, None, 0),
        lambda: L.srdr_body_write_state(None, None, None, 0, 0.0),
        lambda: L.srdr_body_stats(None, None),
        lambda: L.srdr_batch_step(None, 1),
        lambda: L.srdr_batch_info(None, None, None, None, None),
        lambda: L.srdr_batch_mode(None, srdr.SRDR_BATCH_STREAMS),
    ]
    for call in calls:
        assert call() == srdr.SRDR_ERR_INVALID
        assert srdr.last_error()
    # destroying a null handle is a no-op
    L.srdr_body_destroy(None)
    L.srdr_batch_destroy(None)
