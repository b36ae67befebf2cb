"""The Tucker checkpoint's file format on CPU (no GPU, no library call): a file in the format
LatticeSum.save writes is restored field by field by load_checkpoint, and a file of another
format is refused. The GPU round trip through a reduced context is in test_gpu_checkpoint."""
import json

import numpy as np
import pytest

from paper_1411_1994_gb300 import lattice_sum as L


def _write(path, fmt="lattice_sum.tucker.v1"):
    rng = np.random.default_rng(11)
    N, ranks = 12, (3, 4, 2)
    arrays = {f"Z{l}": rng.standard_normal((ranks[l], N)) for l in range(3)}
    arrays["core"] = rng.standard_normal(ranks)
    for l in range(3):
        arrays[f"sigma{l}"] = np.sort(rng.random(5))[::-1]
    arrays["ranks"] = np.asarray(ranks, dtype=np.int32)
    meta = {"format": fmt, "params": {"N": N, "R": 8}, "info": {"r": list(ranks)}, "extra": {"note": "x"}}
    arrays["meta"] = np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8)
    np.savez(path, **arrays)
    return arrays, meta


def test_checkpoint_round_trip_of_the_file_format(tmp_path):
    path = str(tmp_path / "t.npz")
    arrays, meta = _write(path)
    ck = L.load_checkpoint(path)
    assert ck.ranks == [3, 4, 2] and ck.N == 12
    for l in range(3):
        assert np.array_equal(ck.Z[l], arrays[f"Z{l}"])
        assert np.array_equal(ck.sigma[l], arrays[f"sigma{l}"])
    assert np.array_equal(ck.core, arrays["core"])
    assert ck.params == meta["params"] and ck.info == meta["info"] and ck.extra == meta["extra"]
    # the factors are C-contiguous float64, as the device copies and the C ABI take them
    assert all(z.flags["C_CONTIGUOUS"] and z.dtype == np.float64 for z in ck.Z + [ck.core])


def test_checkpoint_of_another_format_is_refused(tmp_path):
    path = str(tmp_path / "bad.npz")
    _write(path, fmt="something.else")
    with pytest.raises(ValueError):
        L.load_checkpoint(path)
