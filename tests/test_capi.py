"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared call."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dm_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2311_06115_gb300 import build

    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dm_[a-z0-9_]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, f"declared but not exported: {sorted(declared - exported)}"


def test_binding_covers_the_abi():
    import paper_2311_06115_gb300 as dm

    for name in _declared():
        assert hasattr(dm, name), f"binding lacks {name}"


def test_library_loads_and_reports_status_strings():
    import paper_2311_06115_gb300 as dm

    dm.load()
    assert dm.dm_status_str(dm.DM_ENOCONV) == "DM_ENOCONV"
    cfg = dm.dm_config_default()
    assert cfg.m_max == 300 and cfg.check_every >= 1


def test_no_gpu_fails_loudly():
    import numpy as np
    import torch

    import paper_2311_06115_gb300 as dm

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(dm.DmError) as e:
        dm.dm_create(np.zeros((8, 3), np.float32))
    assert e.value.status == dm.DM_ECUDA


def test_sm103a_target_only():
    from paper_2311_06115_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_request_footprint_estimate_is_monotone_and_plausible():
    import numpy as np

    import paper_2311_06115_gb300 as dm

    small = dm.dm_request_bytes(np.zeros((10_000, 3), np.float32), leaf_size=512, max_rank=128, k=20)
    big = dm.dm_request_bytes(np.zeros((100_000, 3), np.float32), leaf_size=512, max_rank=128, k=20)
    assert 0 < small < big
    # the bench workload: leaf blocks (157 MB) + P slots (134 MB) + Krylov basis (120 MB) + workspaces
    assert 500e6 < big < 1.5e9


def test_request_footprint_counts_the_point_copies():
    """Points are held as the caller's copy, the centred/scaled copy and the permuted copy
    (4 N d bytes each); from d = 16 on the tree build also holds an FP64 copy (8 N d bytes)."""
    import numpy as np

    import paper_2311_06115_gb300 as dm

    n = 60_000
    kw = dict(leaf_size=256, max_rank=128, k=10)
    hd = dm.dm_request_bytes(np.zeros((n, 784), np.float32), **kw)
    assert hd >= 20 * n * 784
    d15 = dm.dm_request_bytes(np.zeros((n, 15), np.float32), **kw)
    d16 = dm.dm_request_bytes(np.zeros((n, 16), np.float32), **kw)
    assert d16 - d15 >= 8 * n * 16 + 12 * n - 3 * 256  # each buffer rounded up to 256 bytes


def test_serving_rejects_bad_requests_and_state():
    import numpy as np
    import torch

    import paper_2311_06115_gb300 as dm

    pts = np.zeros((100, 3), np.float32)
    with pytest.raises(dm.DmError) as e:
        dm.dm_submit(pts, k=200)  # k >= N
    assert e.value.status == dm.DM_EINVAL
    if not torch.cuda.is_available():
        with pytest.raises(dm.DmError) as e:
            dm.dm_submit(pts, k=5)  # no server running
        assert e.value.status == dm.DM_ESTATE
        with pytest.raises(dm.DmError) as e:
            dm.dm_serve_start()
        assert e.value.status == dm.DM_ECUDA
    with pytest.raises(dm.DmError) as e:
        dm.dm_poll(123456789)
    assert e.value.status == dm.DM_EINVAL


def test_intrinsic_dim_matches_oracle():
    """dm_intrinsic_dim (host computation in the library, no device work) against the
    oracle's d(t) on random descending spectra, bit for bit; argument errors."""
    import numpy as np

    import oracle as O
    import paper_2311_06115_gb300 as dm

    rng = np.random.default_rng(11)
    for _ in range(300):
        k = int(rng.integers(2, 33))
        lam = np.concatenate([[1.0], np.sort(rng.uniform(-0.2, 1.0, k - 1))[::-1]])
        t = int(rng.integers(1, 200))
        delta = float(rng.uniform(1e-6, 0.999))
        assert dm.dm_intrinsic_dim(lam, t, delta) == O.intrinsic_dim(lam, t, delta)
    for bad in [([1.0], 1, 0.5), ([1.0, 0.5], 0, 0.5), ([1.0, 0.5], 1, 0.0), ([1.0, 0.5], 1, 1.0),
                ([1.0, float("nan")], 1, 0.5)]:
        with pytest.raises(dm.DmError) as e:
            dm.dm_intrinsic_dim(*bad)
        assert e.value.status == dm.DM_EINVAL
