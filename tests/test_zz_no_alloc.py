"""The allocation-free noise entry point, for callers that cannot allocate
device memory (their memory belongs to another allocator or a fixed budget).
It must give the same field as mmc_noise, bit for bit (integer-valued Z(4)
entries), on consecutive calls that share its static device table.  This file
is collected last so that a failure here comes after every other test."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mmc():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_00016_gb300 import mmc as m
    return m


def test_noise_noalloc_matches_mmc_noise(mmc):
    import torch
    ctx = mmc.mmc_create((6, 4, 2, 6), seed=123, device=0)
    try:
        # two calls in a row: a large batch, then a smaller one (the table keeps the first call's entries)
        for (level, first, nrhs) in [(3, 17, 37), (5, 2, 5)]:
            for prec in (mmc.MMC_F64, mmc.MMC_F32, mmc.MMC_BF16):
                want = mmc.new_field(ctx, nrhs, prec)
                got = mmc.new_field(ctx, nrhs, prec)
                got.fill_(0x5A)  # garbage: every element must be overwritten
                mmc.mmc_noise(ctx, level, first, mmc.MMC_TAG_NOISE, nrhs, prec, want)
                mmc.mmc_noise_noalloc(ctx, level, first, mmc.MMC_TAG_NOISE, nrhs, prec, got)
                torch.cuda.synchronize()
                assert torch.equal(got, want), (level, first, nrhs, prec)
        # beyond the table: rejected on the host (the field is sized for the request all the same)
        big = mmc.new_field(ctx, 4097, mmc.MMC_BF16)
        with pytest.raises(mmc.MMCError):
            mmc.mmc_noise_noalloc(ctx, 0, 0, mmc.MMC_TAG_NOISE, 4097, mmc.MMC_BF16, big)
    finally:
        mmc.mmc_destroy(ctx)
