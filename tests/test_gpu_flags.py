"""Chained flow launches whose tiles wait for per-tile flags of the previous launch.

A multi-step launch of two to ten waves of CTAs (2048 x 2048 here: 578 to 2052 tiles, depending
on the steps per launch and the tile shape) does not wait for the whole previous launch: each
tile waits for the 3 x 3 tiles of the previous launch whose outputs its window reads and whose
windows cover its own output tile.  Whatever the interleaving of the launches, the result must be
the bits of one step per launch (the configuration the per-step parity tests compare with the
oracle, Sec. V-B, Eq. MCF).  Covered: 2 to 8 steps per launch, both tile shapes, a shorter last
launch of 2 steps (another tile grid: it waits for the whole launch before it) or of 1 step, both
boundary rules, BF16/FP16 storage, U^0 given in the output buffer, a pitch that is staged through
the workspace, repeated calls on one workspace (the flags are cleared by every call), and the
status word (no wait ran out).  And the failure path without a fault: a launch whose tiles wait
for flags that no launch stores gives up after its time limit, reports WMC_ERR_TIMEOUT through the
status word, and leaves the context usable.
"""
import pytest
import torch

from paper_1903_07189_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N = 2048


def wmc():
    from paper_1903_07189_gb300 import wmc as m
    return m


@pytest.fixture(scope="module")
def image():
    return torch.from_numpy(synth.make_image(N, N, seed=11, n_bumps=24, n_shapes=12, sigma=0.05)).to(DEV)


@pytest.mark.parametrize("T,tile", [(2, 1), (3, 1), (4, 1), (5, 1), (8, 1), (4, 2), (8, 2)])
def test_chained_launches_equal_one_step_launches(image, T, tile):
    ref = wmc().denoise(image, 1.0, 0.25, 3 * T + 2, steps_per_launch=1)
    ws = torch.empty(wmc().load().wmc_denoise_workspace_size(N, N, N, 0), dtype=torch.uint8, device=DEV)
    for _ in range(2):  # the second call reuses the flags the first left behind
        got = wmc().denoise(image, 1.0, 0.25, 3 * T + 2, steps_per_launch=T, tile=tile, workspace=ws)
        assert torch.equal(got, ref), (T, tile)
    wmc().check_status(ws)
    # whole launches only (no shorter last launch)
    assert torch.equal(wmc().denoise(image, 1.0, 0.25, 4 * T, steps_per_launch=T, tile=tile),
                       wmc().denoise(image, 1.0, 0.25, 4 * T, steps_per_launch=1))


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_chained_launches_16bit_and_zero(image, dtype, bnd):
    f = image.to(dtype)
    ref = wmc().denoise(f, 1.0, 0.25, 12, bnd, steps_per_launch=1)
    assert torch.equal(wmc().denoise(f, 1.0, 0.25, 12, bnd), ref)


def test_chained_launches_in_place_and_staged(image):
    # U^0 in the output buffer: the first launch writes the workspace, the second the output
    u = image.clone()
    ref = wmc().denoise(image, 1.0, 0.25, 16, steps_per_launch=1)
    wmc().denoise(image, 1.0, 0.25, 16, u0=u, out=u)
    assert torch.equal(u, ref)
    # rows of 2047 elements (not a multiple of 16 bytes): staged through aligned workspace images
    big = torch.zeros((N, N + 1), device=DEV)
    big[:, :N - 1] = image[:, :N - 1]
    f = big[:, :N - 1]
    ref = wmc().denoise(f, 1.0, 0.25, 13, steps_per_launch=1)
    assert torch.equal(wmc().denoise(f, 1.0, 0.25, 13, steps_per_launch=4), ref)


def test_flag_wait_that_runs_out_is_reported(image):
    ws = torch.empty(wmc().load().wmc_denoise_workspace_size(N, N, N, 0), dtype=torch.uint8, device=DEV)
    out = torch.empty_like(image)
    wmc().selftest_flag_timeout(image, out, ws)
    with pytest.raises(wmc().WMCError) as err:
        wmc().check_status(ws)
    assert err.value.status == 5  # WMC_ERR_TIMEOUT
    # the launch went ahead after the wait (its input, f, was ready): 4 steps from f
    assert torch.equal(out, wmc().denoise(image, 1.0, 0.25, 4))
    # the next flow call on the workspace clears the word and gives the exact result
    got = wmc().denoise(image, 1.0, 0.25, 9, workspace=ws)
    wmc().check_status(ws)
    assert torch.equal(got, wmc().denoise(image, 1.0, 0.25, 9, steps_per_launch=1))
