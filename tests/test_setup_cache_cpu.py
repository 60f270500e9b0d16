"""Setup blobs on the host side: the problem key and the checks aim_import_setup makes before any
CUDA call (no GPU here). The round trip through the device is in test_gpu_setup_cache.py.
"""
import math
import struct

import numpy as np
import pytest

import synth

K = 2.0 * math.pi
# header of a setup blob as include/aim.h describes it (little-endian, 160 bytes)
HEADER = struct.Struct("<8sIIQQQ8i5d4i4q")


@pytest.fixture(scope="module")
def aim():
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim


def test_header_layout_is_160_bytes():
    assert HEADER.size == 160


def test_key_is_a_function_of_the_problem(aim):
    nodes = synth.StarContour.from_seed(2).polygon(10.0, 200)
    base = dict(fft_P=0, s=4, quad_p=4, near_radius=0.0, alpha=3.0 * K)
    k0 = aim.setup_key(nodes, K, aim.TE, 64, **base)
    assert k0 == aim.setup_key(nodes.copy(), K, aim.TE, 64, **base)
    assert len(k0) == 16 and int(k0, 16) >= 0
    # the same problem stated another way: fft_P = 0 selects 128 for m = 64
    assert k0 == aim.setup_key(nodes, K, aim.TE, 64, **dict(base, fft_P=128))
    # any change of what the setup depends on changes the key
    moved = nodes.copy()
    moved[17, 0] = np.nextafter(moved[17, 0], np.inf)
    others = [
        aim.setup_key(moved, K, aim.TE, 64, **base),
        aim.setup_key(nodes, np.nextafter(K, 0.0), aim.TE, 64, **base),
        aim.setup_key(nodes, K, aim.TM, 64, **base),
        aim.setup_key(nodes, K, aim.TE, 65, **base),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, fft_P=256)),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, s=5)),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, quad_p=5)),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, near_radius=0.3)),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, alpha=3.5 * K)),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, alpha=None)),
        aim.setup_key(nodes, K, aim.TE, 64, **dict(base, filter_kind=aim.FILTER_ANALYTIC)),
    ]
    assert len(set(others + [k0])) == len(others) + 1


def test_key_checks_its_arguments(aim):
    nodes = synth.circle_polygon(1.0, 64)
    with pytest.raises(aim.AimError) as exc:
        aim.setup_key(nodes, -1.0, aim.TE, 32)
    assert exc.value.status == aim.EINVAL


def _header(**over):
    f = dict(magic=b"AIMSETUP", version=1, header_bytes=160, key=0, payload=0, checksum=0, form=1, n=64, m=32,
             P=64, s=4, p=4, filter_kind=0, nproj=4, k=K, L=1.5, eps=3.0 / 31, alpha=0.0, near_radius=0.5, n_act=1,
             row_lo=0, row_hi=0, gram_band=32, n_sc=0, n_ga=0, n_gram=64 * 64, nnz=0)
    f.update(over)
    return HEADER.pack(f["magic"], f["version"], f["header_bytes"], f["key"], f["payload"], f["checksum"], f["form"],
                       f["n"], f["m"], f["P"], f["s"], f["p"], f["filter_kind"], f["nproj"], f["k"], f["L"], f["eps"],
                       f["alpha"], f["near_radius"], f["n_act"], f["row_lo"], f["row_hi"], f["gram_band"], f["n_sc"],
                       f["n_ga"], f["n_gram"], f["nnz"])


def _import(aim, blob, **kw):
    nodes = synth.circle_polygon(1.0, 64)
    args = dict(L=1.5, near_radius=0.5)
    args.update(kw)
    return aim.Context(nodes, K, aim.TE, 32, blob=np.frombuffer(blob, dtype=np.uint8), **args)


@pytest.mark.parametrize("case", ["short", "magic", "version", "length", "other_k", "other_m", "other_filter"])
def test_import_refuses_a_bad_blob_before_any_cuda_call(aim, case):
    payload = bytes(64)
    blob = {
        "short": b"AIMSETUP",
        "magic": _header(magic=b"NOTSETUP", payload=64) + payload,
        "version": _header(version=2, payload=64) + payload,
        "length": _header(payload=48) + payload,
        "other_k": _header(k=K * 1.5, payload=64) + payload,
        "other_m": _header(m=40, payload=64) + payload,
        "other_filter": _header(filter_kind=1, alpha=3.0 * K, payload=64) + payload,
    }[case]
    with pytest.raises(aim.AimError) as exc:
        _import(aim, blob)
    assert exc.value.status == aim.EINVAL
    reason = str(exc.value)
    expect = {"short": "too short", "magic": "bad magic", "version": "format version", "length": "truncated",
              "other_k": "k differs", "other_m": "m differs", "other_filter": "filter kind differs"}[case]
    assert expect in reason, reason


def test_import_refuses_inconsistent_sizes(aim):
    # every problem parameter matches, but the counts cannot belong to it (a TE blob with one projection)
    payload = bytes(64)
    with pytest.raises(aim.AimError) as exc:
        _import(aim, _header(nproj=1, payload=64) + payload)
    assert exc.value.status == aim.EINVAL and "inconsistent sizes" in str(exc.value)
