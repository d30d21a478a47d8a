"""The FP64 oracle against facts fixed by the paper's definition and by mathematics (CPU only)."""
import numpy as np
import pytest
import torch

import oracle
import oracle_checks as oc


@pytest.mark.parametrize("check", oc.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check, oracle_lib):
    check(oracle_lib)


def _edge_values():
    rng = np.random.default_rng(0)
    special = np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 70000.0, 2.0 ** -24,
                        2.0 ** -25, 3 * 2.0 ** -26, 2.0 ** -14, 1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11,
                        1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, 3.3895e38, 1e-40, np.inf, -np.inf],
                       dtype=np.float32)
    rand = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.uniform(-8, 6, size=20000),
                           rng.uniform(-1, 1, size=20000)]).astype(np.float32)
    return np.concatenate([special, rand])


def test_round_f16_matches_ieee_binary16_cast():
    x = _edge_values()
    got = oracle.round_f16(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float32)  # numpy: IEEE binary16, ties to even
    assert np.array_equal(got, ref)


def test_round_bf16_matches_bfloat16_cast():
    x = _edge_values()
    got = oracle.round_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got, ref)


def test_round_bf16_ties_to_even_by_hand():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (7 fraction bits): ties go to the even 1.0;
    # 1 + 3*2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: the even neighbour is 1 + 2^-6.
    got = oracle.round_bf16(np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8], np.float32))
    assert got.tolist() == [1.0, 1 + 2.0 ** -6]


def test_oracle_rejects_bad_arguments(oracle_lib):
    with pytest.raises(RuntimeError):
        oracle.backproject(4, 3, 3, np.zeros((1, 3, 4)), np.zeros(3), np.ones(3),
                           np.zeros((1, 3, 3), np.float32), z_range=(0, 5))
    # a voxel behind the source (w <= 0) is reported, not silently summed
    mat = np.array([[1.0, 0, 0, 0], [0, 1.0, 0, 0], [0, 0, 0, -1.0]])
    with pytest.raises(RuntimeError):
        oracle.backproject(2, 3, 3, mat[None], np.zeros(3), np.ones(3), np.zeros((1, 3, 3), np.float32))
