"""Proposal-network checkpoint: save and load reproduce the FP32 weights,
Adam's moments and step count exactly, and the BF16 inference copy (CPU)."""
import os

import pytest
import torch

from paper_2404_14044_b300 import hashpoint as H


def test_round_trip(tmp_path):
    st = H.ProposalState("cpu", seed=3)
    g = torch.Generator().manual_seed(5)
    st.m = torch.randn(H.PROP_PARAMS, generator=g)
    st.v = torch.rand(H.PROP_PARAMS, generator=g)
    st.params = st.params + 1e-3 * torch.randn(H.PROP_PARAMS, generator=g)
    st.refresh_bf16()
    st.step = 17
    path = os.path.join(tmp_path, "prop.ckpt")
    st.save(path)
    ld = H.ProposalState.load(path, "cpu")
    assert ld.step == 17
    for name in ("params", "m", "v", "bf16"):
        assert torch.equal(getattr(ld, name), getattr(st, name)), name
    assert torch.equal(ld.grad, torch.zeros(H.PROP_PARAMS))


def test_rejects_bad_files(tmp_path):
    st = H.ProposalState("cpu", seed=0)
    path = os.path.join(tmp_path, "prop.ckpt")
    st.save(path)
    blob = open(path, "rb").read()
    bad = os.path.join(tmp_path, "bad.ckpt")
    open(bad, "wb").write(b"XXXXXXXX" + blob[8:])
    with pytest.raises(ValueError):
        H.ProposalState.load(bad, "cpu")
    open(bad, "wb").write(blob[:-4])                   # truncated arrays
    with pytest.raises(ValueError):
        H.ProposalState.load(bad, "cpu")
