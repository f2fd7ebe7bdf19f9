"""The seeded input generators (CPU): the shapes the join-variant workloads
rely on, since the full-size GPU tests build their expected outputs from them."""
import numpy as np
import torch

from paper_2506_09226_gb300 import datagen


def test_multi_dim_rows_per_key():
    m = datagen.multi_dim(1000, 4, 25, seed=3)
    k = m["key"].numpy()
    assert m["key"].dtype == torch.int32 and len(k) == 4000
    assert np.array_equal(np.bincount(k, minlength=1000), np.full(1000, 4))
    assert not np.array_equal(k, np.sort(k))            # rows in random order
    a = m["attr"].numpy()
    assert a.min() >= 0 and a.max() < 25
    again = datagen.multi_dim(1000, 4, 25, seed=3)
    assert torch.equal(again["key"], m["key"]) and torch.equal(again["attr"], m["attr"])
    e = datagen.multi_dim(0, 4, 25, seed=3)
    assert e["key"].numel() == 0 and e["attr"].numel() == 0


def test_pair_dim_unique_pairs_and_probe():
    p = datagen.pair_dim(500, 4, seed=7)
    hi, lo, off = p["hi"].numpy(), p["lo"].numpy(), p["off"].numpy()
    assert len(hi) == 2000 and p["payload"].numel() == 2000
    assert np.array_equal(np.bincount(hi, minlength=500), np.full(500, 4))
    j = lo - off[hi]
    assert j.min() == 0 and j.max() == 3
    assert len(set(zip(hi.tolist(), lo.tolist()))) == 2000
    assert off.min() >= 0 and off.max() < 2 ** 30
    fk = torch.from_numpy(np.random.default_rng(1).integers(0, 500, 50_000).astype(np.int32))
    plo = datagen.pair_probe_lo(fk, p["off"], 5, seed=7).numpy()
    jj = plo - off[fk.numpy()]
    assert jj.min() == 0 and jj.max() == 4
    # about one probe row in five has no partner
    assert abs((jj == 4).mean() - 0.2) < 0.01
