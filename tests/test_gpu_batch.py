"""Batched sweeps (extension): several films of uneven size swept together
-- as one graph with a branch per problem, as grouped launches, or on a
stream per problem -- give exactly what sweeping each film alone gives
(same kernels, launch shapes and fixed-order reductions), and one of them
matches the CPU oracle's loop."""
import numpy as np
import pytest
import torch

from oracle import micromag as om
from paper_1405_2728_gb300 import inputs
from gpu_cases import dev

pytestmark = pytest.mark.gpu


def small_films():
    films = inputs.batch_films(count=5, seed=77, max_mT=20.0, step_mT=4.0)
    # shrink to quick sizes, keeping the uneven shapes
    out = []
    for w in films:
        w.nx, w.ny = max(8, w.nx // 8), max(4, w.ny // 8)
        w.dx = w.dy = w.dz = 5e-9
        out.append(w)
    return out


KINDS = ["branches", "grouped", "streams"]


def kind_of(mmlib, name):
    return {"branches": mmlib.MM_BATCH_BRANCHES, "grouped": mmlib.MM_BATCH_GROUPED,
            "streams": mmlib.MM_BATCH_STREAMS}[name]


@pytest.mark.parametrize("kind", KINDS)
def test_batch_equals_single_sweeps_and_oracle(mmlib, kind):
    films = small_films()
    probs = [mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz),
                                     mmlib.make_material(w.Ms, w.A, w.K)) for w in films]
    F = films[0].fields()
    opts = mmlib.make_opts(tol=1e-6)
    batch = mmlib.mm_batch_create(probs, kind_of(mmlib, kind))
    assert mmlib.mm_batch_kind(batch) == kind_of(mmlib, kind)
    ms = [dev(w.initial_m()) for w in films]
    st, mavg, res = mmlib.mm_batch_sweep(batch, ms, F, opts=opts)
    assert st == mmlib.MM_OK
    assert all(r.converged for rs in res for r in rs)
    for i, (w, p) in enumerate(zip(films, probs)):
        m1 = dev(w.initial_m())
        st1, mavg1, res1 = mmlib.mm_hysteresis_sweep(p, m1, F, opts=opts)
        assert st1 == mmlib.MM_OK
        assert np.array_equal(mavg[i], mavg1), i
        assert torch.equal(ms[i], m1), i
        assert [r.heff_evals for r in res[i]] == [r.heff_evals for r in res1]
    # the batch's first film against the CPU oracle (loop metrics: switching field within one
    # field step and remanence within 1e-3, since rounding may pick a different branch at switching)
    w = films[0]
    op = om.Problem(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, Ms=w.Ms, A=w.A, K=w.K)
    ref, _, _ = om.sweep(op, w.initial_m(), F, om.Demag(op), tol=1e-6)
    a, b = om.loop_metrics(F, mavg[0]), om.loop_metrics(F, ref)
    step = np.linalg.norm(F[0] - F[1])
    if np.isnan(b["H_sw"]):
        assert np.isnan(a["H_sw"])
    else:
        assert abs(a["H_sw"] - b["H_sw"]) <= step * (1 + 1e-9)
    assert abs(a["M_r"] - b["M_r"]) <= 1e-3
    batch.close()


@pytest.mark.parametrize("kind", KINDS)
def test_batch_fp32_mixed_with_fp64(mmlib, kind):
    # a batch may mix precisions; each member equals its own single sweep
    films = small_films()[:3]
    precs = [mmlib.MM_FP32, mmlib.MM_FP64, mmlib.MM_FP32]
    probs = [mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz),
                                     mmlib.make_material(w.Ms, w.A, w.K), pr) for w, pr in zip(films, precs)]
    dts = [torch.float32 if pr == mmlib.MM_FP32 else torch.float64 for pr in precs]
    F = films[0].fields()[:5]
    opts = mmlib.make_opts(tol=1e-5)
    batch = mmlib.mm_batch_create(probs, kind_of(mmlib, kind))
    ms = [dev(w.initial_m(), dt) for w, dt in zip(films, dts)]
    st, mavg, res = mmlib.mm_batch_sweep(batch, ms, F, opts=opts)
    assert st == mmlib.MM_OK
    for i, (w, p, dt) in enumerate(zip(films, probs, dts)):
        m1 = dev(w.initial_m(), dt)
        st1, mavg1, _ = mmlib.mm_hysteresis_sweep(p, m1, F, opts=opts)
        assert st1 == mmlib.MM_OK
        assert np.array_equal(mavg[i], mavg1), i
        assert torch.equal(ms[i], m1), i
    batch.close()


@pytest.mark.parametrize("kind", ["branches", "streams"])
def test_batch_with_bulk_and_double_word_members_equals_single_sweeps(mmlib, kind):
    """A three-dimensional grid (bulk layout) and a double-word problem may
    join a branch-graph or stream batch (grouped launches refuse them); every
    member still equals its own single sweep bit for bit."""
    films = small_films()[:3]
    cube = inputs.Workload("cube_6", 6, 6, 6, 5e-9, 5e-9, 5e-9, K=2e4)
    members = films + [cube]
    precs = [mmlib.MM_FP64, mmlib.MM_FP64, mmlib.MM_F32X2, mmlib.MM_FP64]
    probs = [mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz),
                                     mmlib.make_material(w.Ms, w.A, w.K), pr) for w, pr in zip(members, precs)]
    assert mmlib.mm_problem_info(probs[-1])["bulk_layout"] == 1
    F = films[0].fields()[:4]
    opts = mmlib.make_opts(tol=1e-6)
    with pytest.raises(mmlib.MMError) as e:
        mmlib.mm_batch_create(probs, mmlib.MM_BATCH_GROUPED)
    assert e.value.status == mmlib.MM_ERR_UNSUPPORTED
    batch = mmlib.mm_batch_create(probs, kind_of(mmlib, kind))
    ms = [dev(w.initial_m()) for w in members]
    st, mavg, res = mmlib.mm_batch_sweep(batch, ms, F, opts=opts)
    assert st == mmlib.MM_OK
    for i, (w, p) in enumerate(zip(members, probs)):
        m1 = dev(w.initial_m())
        st1, mavg1, res1 = mmlib.mm_hysteresis_sweep(p, m1, F, opts=opts)
        assert st1 == mmlib.MM_OK
        assert np.array_equal(mavg[i], mavg1), i
        assert torch.equal(ms[i], m1), i
        assert [r.heff_evals for r in res[i]] == [r.heff_evals for r in res1]
    batch.close()


@pytest.mark.parametrize("kind", ["branches", "grouped"])
def test_graph_batch_repeats_and_resumes(mmlib, kind):
    """Two sweep calls on one batch (the second resuming at a later field
    value, with more field values than the first) give what one sweep gives."""
    films = small_films()[:3]
    probs = [mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz),
                                     mmlib.make_material(w.Ms, w.A, w.K)) for w in films]
    F = films[0].fields()
    opts = mmlib.make_opts(tol=1e-6)
    b1 = mmlib.mm_batch_create(probs, kind_of(mmlib, kind))
    ms1 = [dev(w.initial_m()) for w in films]
    _, mavg1, _ = mmlib.mm_batch_sweep(b1, ms1, F, opts=opts)
    b1.close()
    b2 = mmlib.mm_batch_create(probs, kind_of(mmlib, kind))
    ms2 = [dev(w.initial_m()) for w in films]
    mmlib.mm_batch_sweep(b2, ms2, F[:4], opts=opts)
    _, mavg2, _ = mmlib.mm_batch_sweep(b2, ms2, F, start=4, opts=opts)
    for i in range(len(films)):
        assert np.array_equal(mavg1[i][4:], mavg2[i][4:]), i
        assert torch.equal(ms1[i], ms2[i]), i
    b2.close()


def test_branch_batch_follows_a_member_recapture(mmlib):
    """The branch graph holds each member's kernel parameters: after a member's
    own minimiser graph is recaptured (a per-cell anisotropy set after the batch
    was made), the next sweep call rebuilds the batch graph and the member
    sweeps with its new anisotropy, equal to its own single sweep."""
    films = small_films()[:2]
    probs = [mmlib.mm_setup_geometry(mmlib.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz),
                                     mmlib.make_material(w.Ms, w.A, w.K)) for w in films]
    F = films[0].fields()[:4]
    opts = mmlib.make_opts(tol=1e-6)
    batch = mmlib.mm_batch_create(probs)
    assert mmlib.mm_batch_kind(batch) == mmlib.MM_BATCH_BRANCHES
    ms = [dev(w.initial_m()) for w in films]
    mmlib.mm_batch_sweep(batch, ms, F, opts=opts)
    w = films[1]
    Kc = np.linspace(0.5, 1.5, w.nx * w.ny * w.nz).reshape(w.nz, w.ny, w.nx) * max(w.K, 500.0)
    mmlib.mm_set_anisotropy(probs[1], Kc)
    ms = [dev(w.initial_m()) for w in films]
    st, mavg, _ = mmlib.mm_batch_sweep(batch, ms, F, opts=opts)
    assert st == mmlib.MM_OK
    m1 = dev(w.initial_m())
    st1, mavg1, _ = mmlib.mm_hysteresis_sweep(probs[1], m1, F, opts=opts)
    assert np.array_equal(mavg[1], mavg1)
    assert torch.equal(ms[1], m1)
    batch.close()
