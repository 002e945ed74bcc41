"""Split multigrid sweeps: on a level of at least 2^25 cells (2^23 with a
permittivity field) whose z faces are not periodic, the pre-smoother, the
prolongation sweep and the coarse levels' second post-sweep run as two
launches (interior planes with the face code compiled out, then the two face
slabs).  Each cell goes through the same arithmetic
either way, so a film whose sweeps are split must match, bit for bit, the
same film with every sweep as one launch (pf_tiling.mg_whole = 1)."""
import pytest
import torch

from paper_1202_6116_gb300 import build as B
from paper_1202_6116_gb300 import pf
from paper_1202_6116_gb300 import workloads as W
from paper_1202_6116_gb300.film import Film

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pf.lib()


def _pair(w, steps):
    films = []
    for whole in (0, 1):
        f = Film(w)
        t = pf.pf_get_tiling(f.ctx)
        pf.pf_set_tiling(f.ctx, t.vx, t.tz, t.blocks_per_sm, mg_whole=whole)
        assert pf.pf_get_tiling(f.ctx).mg_whole == whole
        st, info = f.step(steps)
        assert st == pf.PF_OK
        films.append((f, info))
    return films


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_split_sweeps_match_whole_sweeps_tip(precision):
    # 512 x 512 x 128 = 2^25 cells: the finest level splits, the next does not.  In
    # FP32 the finest level's pre-smoother + residual and its two post-sweeps also
    # run fused; the post-sweeps' r.z is then summed over the interior and the face
    # slabs' tiles in another order and rounded in another grouping, so FP32 is
    # compared within the solve tolerance, FP64 (nothing fused) bit for bit.
    w = W.film_tip_fp32(512, 512, 128, seed=3).with_(solver="mg", maxit=500, precision=precision,
                                                      rtol=1e-7 if precision == "fp32" else 1e-10)
    (a, ia), (b, ib) = _pair(w, 4)
    if precision == "fp64":
        assert torch.equal(a.P, b.P) and torch.equal(a.phi, b.phi)
        assert ia["total_iters"] == ib["total_iters"]
    else:
        for x, y in ((a.P, b.P), (a.phi, b.phi)):
            scale = float(y.abs().max())
            assert float((x - y).abs().max()) <= 1e-5 * scale
        assert abs(ia["total_iters"] - ib["total_iters"]) <= 4
    assert ia["solves"] == ib["solves"] == 4
    extra = ia["kernel_launches"] - ib["kernel_launches"]
    assert extra > 0 and extra % 2 == 0          # two more launches per V-cycle
    a.close()
    b.close()


def test_fused_finest_level_matches_oracle_grade_solve():
    """The fused finest-level passes (FP32 tip film, 2^25 cells) solve the
    potential to the requested tolerance: the true residual of the solved
    potential, formed in FP64 on the device, stays within a small factor of it."""
    w = W.film_tip_fp32(512, 512, 128, seed=3).with_(solver="mg", maxit=500)
    f = Film(w)
    st, info = f.step(6)
    assert st == pf.PF_OK and info["nonconverged"] == 0
    Pprev = f.P.clone()                  # the state the next step's solve is for
    st, info = f.step(1)
    assert st == pf.PF_OK and info["last_relres"] < w.rtol
    stored, bnorm, comp = f.true_residual(Pprev)
    assert comp / bnorm < 10 * w.rtol
    f.close()


@pytest.mark.parametrize("shape", [(528, 512, 128), (512, 512, 129)])
def test_split_fallbacks_match_whole_sweeps(shape):
    """Shapes the fused finest-level passes do not take whole: nx not a multiple
    of the 64-column tile (split sweeps only), and an odd nz (no z coarsening on
    the finest level: the fused pre-smoother + residual restricts plane by plane,
    the post-sweeps stay unfused).  Bit for bit against whole-level sweeps."""
    w = W.film_tip_fp32(*shape, seed=4).with_(solver="mg", maxit=500)
    (a, ia), (b, ib) = _pair(w, 3)
    assert torch.equal(a.P, b.P) and torch.equal(a.phi, b.phi)
    assert ia["total_iters"] == ib["total_iters"]
    assert ia["kernel_launches"] > ib["kernel_launches"]
    a.close()
    b.close()


def test_split_sweeps_match_whole_sweeps_open_air():
    # permittivity field, open top face, 512 x 512 x 37 > 2^23 cells: the eps sweeps split
    w = W.film_open_air(512, 512, 37, seed=5).with_(solver="mg", maxit=500)
    (a, ia), (b, ib) = _pair(w, 2)
    assert torch.equal(a.P, b.P) and torch.equal(a.phi, b.phi)
    assert ia["total_iters"] == ib["total_iters"]
    assert ia["kernel_launches"] > ib["kernel_launches"]
    a.close()
    b.close()


def test_mg_whole_is_validated():
    w = W.film_tip_fp32(32, 32, 8, seed=3).with_(solver="mg")
    f = Film(w)
    t = pf.pf_get_tiling(f.ctx)
    with pytest.raises(pf.PfError) as e:
        pf.pf_set_tiling(f.ctx, t.vx, t.tz, t.blocks_per_sm, mg_whole=2)
    assert e.value.status == pf.PF_ERR_ARG
    f.close()
