"""Largest-size case: AX over more than 2^31 points (64-bit point offsets).

nx = 16 and 524 352 elements give 2 147 745 792 points.  Every element gets the
geometric factors of one deformed element (the operator does not care), u is
random, and sampled elements on both sides of the 2^31 boundary are compared
with the oracle.  Native FP64 (G: 103 GB) and float-float (Gff: 103 GB) run one
after the other, each with u and w (17 GB each) on the device.  Skipped on a
GPU with less than 200 GB.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import ref  # noqa: E402
from paper_2011_04981_gb300 import inputs, nekax  # noqa: E402

DEV = "cuda"
NX = 16
NELT = (1 << 31) // NX ** 3 + 64


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available() or torch.cuda.get_device_properties(0).total_memory < 200e9:
        pytest.skip("needs a GPU with at least 200 GB")
    nekax.load()
    torch.cuda.empty_cache()  # memory cached by earlier tests of the session
    mesh = inputs.box_mesh(2, 2, 2, NX, perturb=0.2, seed=5)  # the centre vertex moves: deformed elements
    xi, rho, D = ref.gll(NX)
    G1 = ref.geom(mesh.corners[:1], NX, xi, rho)[0]  # [N3][6] of one deformed element
    gen = torch.Generator(device=DEV)
    gen.manual_seed(11)
    u = torch.rand((NELT, NX ** 3), dtype=torch.float64, device=DEV, generator=gen)
    u.mul_(2.0).sub_(1.0)
    assert u.numel() > (1 << 31)
    yield D, G1, u
    del u
    torch.cuda.empty_cache()


def _check(w, u, D, G1):
    for e in (0, (1 << 31) // NX ** 3 - 1, (1 << 31) // NX ** 3, NELT - 1):
        ue = u[e].cpu().numpy()[None]
        ref_w = ref.ax(D, G1[None], ue)[0]
        got = w[e].cpu().numpy()
        assert np.max(np.abs(got - ref_w)) <= 1e-12 * np.max(np.abs(ref_w)), e


def test_ax_fp64_beyond_2_31_points(big):
    D, G1, u = big
    G = torch.from_numpy(G1).to(DEV).unsqueeze(0).expand(NELT, -1, -1).contiguous()
    w = torch.empty_like(u)
    nekax.ax(NELT, NX, torch.from_numpy(D).to(DEV), G, u, w)
    torch.cuda.synchronize()
    del G
    _check(w, u, D, G1)
    del w
    torch.cuda.empty_cache()


def test_ax_ff_beyond_2_31_points(big):
    D, G1, u = big
    g1 = torch.from_numpy(G1).to(DEV).reshape(1, NX ** 3, 6).contiguous()
    gff1 = torch.empty((1, NX ** 3, 12), dtype=torch.float32, device=DEV)
    nekax.geom_ff(1, NX, g1, gff1)
    Gff = gff1.expand(NELT, -1, -1).contiguous()
    w = torch.empty_like(u)
    nekax.ax_ff(NELT, NX, torch.from_numpy(D).to(DEV), Gff, u, w)
    torch.cuda.synchronize()
    del Gff
    _check(w, u, D, G1)
    del w
    torch.cuda.empty_cache()
