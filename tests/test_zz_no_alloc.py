"""pic_field_solve_static, the allocation-free field solve (§2 step 2, reading C-23), for
callers that cannot allocate device memory (a caching allocator holding the device's free
memory, paths that must not call cudaMalloc, plug-ins without an allocator), against the
simulation handle's field solve (pic_solve_field / pic_get_grid) and, at the largest grid its
static scratch holds, against the FP64 oracle.

Against a PIC_FP64 handle both sides sum the same exact int128 Green's-function terms and
round the same FP64 operations in the same order, so the bar is bit-identical phi and E; the
relative tolerance 2^-50 of the field's scale is asserted first so a failure reports its
size.  A PIC_FP32 handle multiplies by rounded reciprocals where this entry point divides:
the bar there is one unit in the last place.  Collected last (file name) so it also runs
after every other GPU test in the same process.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2109_04469_gb300 import pic, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL_TOL = 2.0**-50


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2109_04469_gb300 import build as B

    B.build()
    O.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _check(got_phi, got_E, want_phi, want_E, where):
    for name, g, w in (("phi", got_phi, want_phi), ("E", got_E, want_E)):
        scale = max(float(np.max(np.abs(w))), 1e-300)
        assert float(np.max(np.abs(g - w))) <= REL_TOL * scale, (where, name)
        assert np.array_equal(g, w), (where, name, int(np.count_nonzero(g != w)))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_two_calls_in_a_row_match_the_handle_solve():
    cfg = workloads.params("ccp_5pa_150v_128c")
    nc, nx = cfg["n_cells"], cfg["n_cells"] + 1
    sim = pic.Simulation(cfg)
    grids = []
    for n in (25, 7):  # two different charge states and drive phases
        sim.step(n)
        sim.sync()
        g = sim.grid()  # counts of the current step and the field solved from them
        assert np.any(g["Ci"] != g["Ce"])
        grids.append(g)
    ins, outs = [], []
    for g in grids:
        ins.append((_dev(g["Ce"]), _dev(g["Ci"])))
        outs.append((torch.full((nx,), float("nan"), dtype=torch.float64, device="cuda"),
                     torch.full((nx,), float("nan"), dtype=torch.float64, device="cuda")))
    # both calls enqueued back to back on one stream, reusing the static scratch in order
    for g, (ce, ci), (phi, E) in zip(grids, ins, outs):
        V = float(g["phi"][0])  # phi_0 is the drive voltage of that step, exactly
        rc = pic.field_solve_static(ce, ci, nc, cfg["gap_m"], cfg["weight"], cfg["area_m2"],
                                    V, phi, E)
        assert rc == 0
    torch.cuda.synchronize()
    for k, (g, (phi, E)) in enumerate(zip(grids, outs)):
        _check(phi.cpu().numpy(), E.cpu().numpy(), g["phi"], g["E"], f"call {k}")
    sim.close()


def test_fp32_handle_field_within_one_ulp():
    """A PIC_FP32 handle solves the same exact sums but multiplies by the reciprocals of
    N dx, 2 N dx and N; each of phi and E then differs from the divided value by at most
    one unit in the last place."""
    cfg = workloads.params("ccp_5pa_150v_128c", precision=pic.PIC_FP32)
    nc, nx = cfg["n_cells"], cfg["n_cells"] + 1
    sim = pic.Simulation(cfg)
    phi = torch.empty(nx, dtype=torch.float64, device="cuda")
    E = torch.empty(nx, dtype=torch.float64, device="cuda")
    for n in (25, 7):
        sim.step(n)
        sim.sync()
        g = sim.grid()
        rc = pic.field_solve_static(_dev(g["Ce"]), _dev(g["Ci"]), nc, cfg["gap_m"],
                                    cfg["weight"], cfg["area_m2"], float(g["phi"][0]), phi, E)
        assert rc == 0
        torch.cuda.synchronize()
        for name, got, want in (("phi", phi.cpu().numpy(), g["phi"]), ("E", E.cpu().numpy(),
                                                                      g["E"])):
            ulp = np.maximum(np.spacing(np.abs(got)), np.spacing(np.abs(want)))
            assert np.all(np.abs(got - want) <= ulp), (name, n)
    sim.close()


def test_largest_grid_matches_the_oracle():
    nc = pic.FIELD_STATIC_MAX_CELLS
    nx = nc + 1
    cfg = workloads.params("ccp_5pa_150v_128c", n_cells=nc, init_per_species=0,
                           capacity_per_species=64)
    ref = O.OracleSim(cfg)
    rng = np.random.default_rng(65536)
    # counts of about 30 superparticles per node with a net ion excess, in units of 2^-32
    Ce = rng.integers(0, 60 * 2**32, nx, dtype=np.int64)
    Ci = rng.integers(0, 64 * 2**32, nx, dtype=np.int64)
    ref.set_counts(Ce, Ci)
    ref.solve_field()  # step 0: V = V_rf cos 0 = V_rf
    r = ref.grid()
    phi = torch.empty(nx, dtype=torch.float64, device="cuda")
    E = torch.empty(nx, dtype=torch.float64, device="cuda")
    for k in range(2):
        pic.field_solve_static(_dev(Ce), _dev(Ci), nc, cfg["gap_m"], cfg["weight"],
                               cfg["area_m2"], cfg["v_rf_amp_v"], phi, E)
        torch.cuda.synchronize()
        _check(phi.cpu().numpy(), E.cpu().numpy(), r["phi"], r["E"], f"call {k}")


def test_sizes_beyond_the_static_scratch_are_rejected():
    nc = pic.FIELD_STATIC_MAX_CELLS + 1
    z = torch.zeros(nc + 1, dtype=torch.int64, device="cuda")
    out = torch.zeros(nc + 1, dtype=torch.float64, device="cuda")
    out2 = torch.zeros(nc + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.field_solve_static(z, z, nc, 0.025, 1.0, 1e-4, 1.0, out, out2)
    assert e.value.code == -7
    assert not torch.any(out != 0) and not torch.any(out2 != 0)
    with pytest.raises(pic.PicError) as e:  # N < 2
        pic.field_solve_static(z, z, 1, 0.025, 1.0, 1e-4, 1.0, out, out2)
    assert e.value.code == -1
