"""lq_dslash_apply_noalloc, the hopping term for callers that cannot allocate
device memory (their own pool owns the GPU, a fixed memory budget, or no
room for the synchronisation a cudaMalloc implies): it must give what
lq_dslash_apply gives, twice in a row on the shared scratch array, and refuse
lattices whose packed fields do not fit in that array.

Collected last (file name) so that a run stopping at its first failure has
run every other test already; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from helpers import TOL, ensure_library, parity_mask, rel_err
from paper_2201_09004_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    ensure_library()
    from paper_2201_09004_b300 import lib
    return lib


def make(L, dims, action, recon):
    lat = L.Lattice(dims)
    if action == "wilson":
        lat.load_gauge(L.THIN, synth.thin_links(dims, 61).cuda())
        return lat, L.op_params(L.WILSON_TM, 0.1, 0.05, recon=recon), 12
    lat.load_gauge(L.FAT, synth.fat_links(dims, 62).cuda())
    lat.load_gauge(L.LONG, synth.long_links(dims, 63).cuda())
    return lat, L.op_params(L.HISQ, 0.05, recon=recon), 3


# (precision, link compression): FP64 always reads R18 links; FP32 and FP16 take R8, R12, R18
PREC_RECON = [(0, 18), (1, 8), (1, 12), (1, 18), (2, 8), (2, 12), (2, 18)]


@pytest.mark.parametrize("action", ["wilson", "hisq"])
@pytest.mark.parametrize("prec,recon", PREC_RECON)
@pytest.mark.parametrize("dagger", [False, True])
def test_noalloc_matches_dslash_apply_twice(L, action, prec, recon, dagger):
    """Two calls in a row (both parities) give what lq_dslash_apply gives with the
    same operator, which also packs the links the no-allocation call needs."""
    import torch
    dims = (8, 8, 8, 16)
    lat, op, ncomp = make(L, dims, action, recon)
    mask = parity_mask(dims)
    for call, parity in enumerate((0, 1)):
        psi = synth.gaussian_field(dims, 70 + call, ncomp=ncomp).cuda()
        ref = lat.dslash_apply(op, parity, psi, dagger=dagger, prec=prec)  # the existing entry point
        out = torch.full_like(psi, complex(7.0, -3.0))                      # stale values must not survive
        lat.dslash_apply_noalloc(op, parity, psi, out, dagger=dagger, prec=prec)
        got, exp = out.cpu().numpy(), ref.cpu().numpy()
        sel = mask == parity
        assert np.all(got[~sel] == 0)
        assert rel_err(got[sel], exp[sel]) <= TOL[prec], (action, prec, recon, dagger, call)


def test_noalloc_binding_checks_sizes_before_the_call(L):
    """The binding refuses tensors of the wrong size, dtype or place before the
    library could write past them."""
    import torch
    dims = (4, 4, 4, 8)
    lat, op, ncomp = make(L, dims, "wilson", 12)
    psi = synth.gaussian_field(dims, 75).cuda()
    lat.dslash_apply(op, 0, psi, prec=L.F32)
    for bad in (torch.zeros(psi.numel() - 12, dtype=torch.complex128, device="cuda"),
                torch.zeros_like(psi, dtype=torch.complex64),
                torch.zeros_like(psi, device="cpu")):
        with pytest.raises(ValueError):
            lat.dslash_apply_noalloc(op, 0, psi, bad, prec=L.F32)


def test_noalloc_rejects_lattice_beyond_the_scratch_size(L):
    import torch
    dims = (24, 24, 24, 32)  # FP64 Wilson packed fields need about 85 MB > 32 MiB
    lat = L.Lattice(dims)
    op = L.op_params(L.WILSON_TM, 0.1, 0.05)
    psi = torch.zeros((32, 24, 24, 24, 4, 3), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    with pytest.raises(L.LqError) as e:
        lat.dslash_apply_noalloc(op, 0, psi, out, prec=L.F64)
    assert e.value.code == L.LQ_EINVAL
    assert "too large" in str(e.value)
