"""The radix-16 DFT stage on CUDA cores and on tensor cores (aim_dft_stage) computes the map its
header states, to the accuracy each arithmetic allows.

The pass maps element i of column c (value c + 256 i of a group of 4096) to output k of column c
(value 16 c + k): X_k(c) = sum_i x_i(c) t(c, i) exp(-2 pi j k i/16), t(c, i) =
exp(-2 pi j (c mod 16) i/256)/4. The reference below applies that definition in FP64. The
CUDA-core butterfly and the split-TF32 tensor-core product are FP32-accurate; plain TF32 operands
are not (the tensor core reads the top 19 bits of each FP32 value: about 2^-10 per operand), which
is why the split is the variant that could replace the butterflies of the complex64 grid product.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GROUP = 4096


@pytest.fixture(scope="module")
def aimlib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2606_10784_gb300 import aim
    return aim


def stage_reference(x: np.ndarray, passes: int) -> np.ndarray:
    """The pass of aim_dft_stage applied `passes` times to each group of 4096 values (FP64)."""
    c = np.arange(256)[:, None]
    i = np.arange(16)[None, :]
    t = np.exp(-2j * np.pi * (c % 16) * i / 256) / 4
    F = np.exp(-2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)   # F[k, i]
    y = x.astype(np.complex128).reshape(-1, GROUP)
    for _ in range(passes):
        cols = y.reshape(-1, 16, 256).transpose(0, 2, 1)          # [group, c, i] = value c + 256 i
        X = np.einsum("gci,ki->gck", cols * t[None], F)           # [group, c, k]
        y = X.reshape(-1, GROUP)                                  # value 16 c + k
    return y.reshape(x.shape)


def run(aim, variant, x, passes):
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    aim.dft_stage(variant, xd, yd, passes)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def inputs(groups, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(groups * GROUP) + 1j * rng.standard_normal(groups * GROUP)).astype(np.complex64)


@pytest.mark.parametrize("passes", [1, 2, 5])
def test_cuda_core_stage_matches_the_definition(aimlib, passes):
    x = inputs(3, passes)
    got = run(aimlib, aimlib.DFT_STAGE_CUDA_CORES, x, passes)
    assert rel(got, stage_reference(x, passes)) < 1e-6 * passes


@pytest.mark.parametrize("passes", [1, 2, 5])
def test_split_tf32_tensor_core_stage_matches_the_definition(aimlib, passes):
    x = inputs(3, 10 + passes)
    got = run(aimlib, aimlib.DFT_STAGE_MMA_TF32X3, x, passes)
    assert rel(got, stage_reference(x, passes)) < 2e-6 * passes


def test_plain_tf32_tensor_core_stage_has_tf32_accuracy(aimlib):
    x = inputs(2, 21)
    want = stage_reference(x, 1)
    err = rel(run(aimlib, aimlib.DFT_STAGE_MMA_TF32, x, 1), want)
    # right map (the error is TF32 rounding, not a wrong entry), but far above FP32 rounding
    assert 1e-5 < err < 4e-3


def test_split_data_path_variant_applies_the_twiddles_in_place(aimlib):
    """Variant 3 (the tensor-core variants' loads, twiddles, operand split and stores without the
    products) stores hi + lo = t(c, i) x_i(c) at value c + 256 i (the split itself is exact)."""
    x = inputs(2, 31)
    c = np.arange(256)[None, :]
    i = np.arange(16)[:, None]
    t = (np.exp(-2j * np.pi * (c % 16) * i / 256) / 4).reshape(-1)    # [i, c] -> value c + 256 i
    want = x.astype(np.complex128).reshape(-1, GROUP)
    for passes in (1, 2):
        want = want * t[None]
        got = run(aimlib, aimlib.DFT_STAGE_SPLIT_ONLY, x, passes)
        assert rel(got, want.reshape(-1)) < 1e-6 * passes


def test_zero_passes_copy_and_every_group_is_independent(aimlib):
    x = inputs(4, 5)
    for v in (0, 1, 2, 3):
        assert np.array_equal(run(aimlib, v, x, 0), x)
    # a group's result does not depend on the others
    x2 = x.copy()
    x2[GROUP:2 * GROUP] = 0
    for v in (0, 2):
        a, b = run(aimlib, v, x, 3), run(aimlib, v, x2, 3)
        assert np.array_equal(a[:GROUP], b[:GROUP]) and np.array_equal(a[2 * GROUP:], b[2 * GROUP:])
        assert not np.any(b[GROUP:2 * GROUP])


def test_in_place_stage(aimlib):
    x = inputs(2, 8)
    xd = torch.from_numpy(x).cuda()
    aimlib.dft_stage(aimlib.DFT_STAGE_CUDA_CORES, xd, xd, 2)
    torch.cuda.synchronize()
    assert np.array_equal(xd.cpu().numpy(), run(aimlib, aimlib.DFT_STAGE_CUDA_CORES, x, 2))


def test_stage_rejects_bad_arguments(aimlib):
    xd = torch.zeros(GROUP, dtype=torch.complex64, device="cuda")
    with pytest.raises(aimlib.AimError) as e:
        aimlib.dft_stage(4, xd, xd, 1)
    assert e.value.status == aimlib.EINVAL
    host = torch.zeros(GROUP, dtype=torch.complex64)
    with pytest.raises(aimlib.AimError) as e:
        aimlib.dft_stage(0, host, xd, 1)
    assert e.value.status == aimlib.EINVAL
    with pytest.raises(aimlib.AimError) as e:
        aimlib.dft_stage(0, xd, xd, -1)
    assert e.value.status == aimlib.EINVAL
