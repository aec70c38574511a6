"""The allocation-free noise entry point, for callers that cannot allocate
device memory (their memory belongs to another allocator or a fixed budget).
It must give the same field as mmc_noise, bit for bit (integer-valued Z(4)
entries), on consecutive calls that share its static device table, and it must
not allocate: it is called first on a fresh context (before mmc_noise has made
that context's own table), and the device's free memory is the same before and
after its calls.  This file is collected last so that a failure here comes after
every other test."""
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
        cases = [(3, 17, 37), (5, 2, 5)]
        fields = {}
        for (level, first, nrhs) in cases:
            for prec in (mmc.MMC_F64, mmc.MMC_F32, mmc.MMC_BF16):
                fields[(level, prec, "got")] = mmc.new_field(ctx, nrhs, prec)
                fields[(level, prec, "want")] = mmc.new_field(ctx, nrhs, prec)
                fields[(level, prec, "got")].fill_(0x5A)  # garbage: every element must be overwritten
        torch.cuda.synchronize()
        # the first call of the process may load the library's device code; from then on
        # no call may change the device's free memory
        level, first, nrhs = cases[0]
        mmc.mmc_noise_noalloc(ctx, level, first, mmc.MMC_TAG_NOISE, nrhs, mmc.MMC_F64,
                              fields[(level, mmc.MMC_F64, "got")])
        free0 = torch.cuda.mem_get_info(0)[0]
        for (level, first, nrhs) in cases:
            for prec in (mmc.MMC_F64, mmc.MMC_F32, mmc.MMC_BF16):
                mmc.mmc_noise_noalloc(ctx, level, first, mmc.MMC_TAG_NOISE, nrhs, prec,
                                      fields[(level, prec, "got")])
                assert torch.cuda.mem_get_info(0)[0] == free0, (level, prec)
        for (level, first, nrhs) in cases:
            for prec in (mmc.MMC_F64, mmc.MMC_F32, mmc.MMC_BF16):
                mmc.mmc_noise(ctx, level, first, mmc.MMC_TAG_NOISE, nrhs, prec, fields[(level, prec, "want")])
        torch.cuda.synchronize()
        for (level, first, nrhs) in cases:
            for prec in (mmc.MMC_F64, mmc.MMC_F32, mmc.MMC_BF16):
                assert torch.equal(fields[(level, prec, "got")], fields[(level, prec, "want")]), (level, prec)
        # beyond the table: rejected on the host (the field is sized for the request all the same)
        big = mmc.new_field(ctx, 4097, mmc.MMC_BF16)
        with pytest.raises(mmc.MMCError):
            mmc.mmc_noise_noalloc(ctx, 0, 0, mmc.MMC_TAG_NOISE, 4097, mmc.MMC_BF16, big)
    finally:
        mmc.mmc_destroy(ctx)
