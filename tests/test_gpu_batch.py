"""Batched stepping: many lattices advanced by one kernel launch per step.

- A batched step gives bit for bit the populations (and FP64 totals) of each
  member stepped alone with the same tile: the batch only changes which block
  works on which lattice, not the arithmetic at any node.
- Replaying the steps as a CUDA graph changes nothing either.
- The autotuner's trial steps are real steps and tile choice never changes the
  populations, so after it the members equal lone engines stepped as often.
- An FP64 batch member matches the FP64 oracle within the parity tolerance.
- Mismatched members, a member stepped alone (parity drift) and parameter
  changes after the batch was made are handled as the header states.
"""
import numpy as np
import pytest

import oracle
import paper_1511_02155_gb300 as tl
from paper_1511_02155_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _well(nx, ny, seed):
    width = 12 + (seed * 7) % (nx // 3)
    depth = 6 + (seed * 5) % (ny // 4)
    return W.square_well(nx, ny, width=width, depth=depth, floor=5)


def _members(kind, prec):
    """(lattice, shape, C, solid, kappa, h) of three unlike lattices of one kind."""
    out = []
    if kind == "wells":
        for s, (nx, ny) in enumerate(((96, 48), (130, 70), (64, 64))):
            C, solid = _well(nx, ny, s + 1)
            kap = (0.01, 0.012 + 0.002 * s, 0.015)
            h = (0.0004 - 0.0002 * s, -0.0003, 0.0002 * s)
            out.append((9, (nx, ny, 1), C, solid, kap, h))
    elif kind == "lens":
        for s, (nx, ny) in enumerate(((96, 80), (150, 64), (64, 33))):
            C = W.lens(nx, ny, 10.0 + 2 * s, 1.0, ny / 4, 3 * ny / 4, (nx / 2, 3 * ny / 4))
            out.append((9, (nx, ny, 1), C, None, (0.01, 0.02 - 0.003 * s, 0.03), (0, 0, 0)))
    elif kind == "spinodal3d":
        for s, (nx, ny, nz) in enumerate(((40, 24, 20), (33, 17, 9), (64, 8, 12))):
            C = W.spinodal((nz, ny, nx), seed=10 + s, amp=0.2)
            out.append((19, (nx, ny, nz), C, None, (0.01, 0.01 + 0.004 * s, 0.02), (0, 0, 0)))
    elif kind == "walls3d":
        for s, (nx, ny, nz) in enumerate(((40, 20, 12), (35, 14, 9))):
            solid = np.zeros((nz, ny, nx), np.uint8)
            solid[:, 0, :] = 1
            solid[:, ny - 1, :] = 1
            solid[2:5, 1:3, 5:9 + s] = 1
            C = W.spinodal((nz, ny, nx), seed=20 + s, amp=0.2)
            out.append((19, (nx, ny, nz), C, solid, (0.01, 0.02, 0.015), (0.0004, -0.0002 * s, 0.0001)))
    return out


def _engine(Q, shape, C, solid, kap, h, prec):
    nx, ny, nz = shape
    eng = tl.TernaryLB(Q, nx, ny, nz, kap, 1.0, 1.0, 0.1, 0.1, h,
                       None if solid is None else solid.reshape(-1), prec)
    rho, phi, psi = W.to_aux(*C)
    if solid is not None:
        for a in (rho, phi, psi):
            a[solid.reshape(a.shape) != 0] = 0.0
    eng.init_fields(rho, phi, psi)
    return eng


def _pairs(kind, prec):
    specs = _members(kind, prec)
    batched = [_engine(*sp, prec) for sp in specs]
    lone = [_engine(*sp, prec) for sp in specs]
    return batched, lone


CASES = [("wells", "fp32"), ("wells", "fp16"), ("wells", "fp64"), ("lens", "fp32"), ("lens", "bf16"),
         ("spinodal3d", "fp32"), ("spinodal3d", "fp16"), ("spinodal3d", "fp64"), ("walls3d", "fp32"),
         ("walls3d", "fp64")]


@pytest.mark.parametrize("kind,prec", CASES)
def test_batch_equals_lone_engines_bitwise(kind, prec):
    batched, lone = _pairs(kind, prec)
    with tl.TernaryBatch(batched) as b:
        b.step(7)
        for e in lone:
            e.step(7)
        for eb, el in zip(batched, lone):
            assert eb.steps_done == 7
            assert np.array_equal(eb.get_populations(), el.get_populations())
            assert np.array_equal(eb.step_mass(), el.step_mass())
            assert np.array_equal(eb.mass(), el.mass())


@pytest.mark.parametrize("kind,prec", [("wells", "fp32"), ("spinodal3d", "fp16")])
def test_graph_replay_equals_plain_batch(kind, prec):
    a, b_ = _pairs(kind, prec)
    with tl.TernaryBatch(a) as plain, tl.TernaryBatch(b_) as graph:
        graph.set_graph(True)
        for n in (9, 1, 4, 3):  # odd counts leave the graph at the other parity
            plain.step(n)
            graph.step(n)
        for ea, eb in zip(a, b_):
            assert ea.steps_done == eb.steps_done == 17
            assert np.array_equal(ea.get_populations(), eb.get_populations())
            assert np.array_equal(ea.step_mass(), eb.step_mass())


@pytest.mark.parametrize("kind,prec", [("wells", "fp32"), ("lens", "fp32")])
def test_autotune_advances_members_without_changing_results(kind, prec):
    batched, lone = _pairs(kind, prec)
    with tl.TernaryBatch(batched) as b:
        variant, chunk = b.autotune(trial_steps=2)
        assert 0 <= variant <= 3 and chunk in (0, 16, 32, 64)
        n = batched[0].steps_done
        assert n > 0 and all(e.steps_done == n for e in batched)
        b.step(3)
        for e in lone:
            e.step(n + 3)
        for eb, el in zip(batched, lone):
            assert np.array_equal(eb.get_populations(), el.get_populations())


def test_fp64_batch_member_matches_oracle():
    specs = _members("wells", "fp64")[:2]
    engines = [_engine(*sp, "fp64") for sp in specs]
    with tl.TernaryBatch(engines) as b:
        b.set_graph(True)
        b.step(60)
    for (Q, shape, C, solid, kap, h), eng in zip(specs, engines):
        nx, ny, nz = shape
        p = oracle.make_params(Q, nx, ny, nz, kap, 1.0, 1.0, 0.1, 0.1, h)
        rho, phi, psi = W.to_aux(*C)
        for a in (rho, phi, psi):
            a[solid != 0] = 0.0
        pops = oracle.init_equilibrium(p, rho, phi, psi, solid=solid.reshape(-1))
        oracle.step(p, *pops, 60, solid.reshape(-1))
        P = eng.get_populations()
        for s in range(3):
            scale = max(np.abs(pops[s]).max(), 1.0)
            assert np.abs(P[s] - pops[s]).max() / scale <= 1e-12


def test_parameter_change_after_creation_is_seen():
    batched, lone = _pairs("wells", "fp32")
    with tl.TernaryBatch(batched) as b:
        b.set_graph(True)
        b.step(4)
        for e in lone:
            e.step(4)
        batched[1].set_gamma(0.5, 2.0)
        lone[1].set_gamma(0.5, 2.0)
        b.step(4)
        for e in lone:
            e.step(4)
        for eb, el in zip(batched, lone):
            assert np.array_equal(eb.get_populations(), el.get_populations())


def test_batch_rejects_mismatched_members_and_parity_drift():
    w = _pairs("wells", "fp32")[0]
    l3 = _pairs("spinodal3d", "fp32")[0]
    lens = _pairs("lens", "fp32")[0]
    with pytest.raises(tl.TLBMError):
        tl.TernaryBatch([w[0], l3[0]])  # lattices differ
    with pytest.raises(tl.TLBMError):
        tl.TernaryBatch([w[0], lens[0]])  # solid and periodic
    with pytest.raises(tl.TLBMError):
        tl.TernaryBatch([w[0], w[0]])  # the same engine twice
    f16 = _pairs("wells", "fp16")[0]
    with pytest.raises(tl.TLBMError):
        tl.TernaryBatch([w[0], f16[0]])  # precisions differ
    with tl.TernaryBatch(w) as b:
        b.step(1)
        w[0].step(1)  # alone: parity now differs from the others
        with pytest.raises(tl.TLBMError):
            b.step(1)
        w[0].step(1)  # even number of lone steps: back in step
        b.step(2)
        assert [e.steps_done for e in w] == [5, 3, 3]


def test_periodic_tile_without_a_batched_kernel_is_refused():
    engines = _pairs("spinodal3d", "fp32")[0]
    with tl.TernaryBatch(engines) as b:
        blocks = b.blocks
        with pytest.raises(tl.TLBMError):
            b.set_tile(1, 0)  # 32x8 has no batched kernel
        assert b.blocks == blocks  # previous tile kept
        b.set_tile(0, 1)  # one plane per block
        assert b.blocks > blocks
        b.step(2)


@pytest.mark.parametrize("variant,chunk", [(0, 0), (2, 0), (3, 16), (1, 5)])
def test_single_member_batch_at_every_solid_tile_equals_lone_engine(variant, chunk):
    batched, lone = _pairs("wells", "fp32")
    with tl.TernaryBatch(batched[1:2]) as b:
        b.set_tile(variant, chunk)
        b.set_graph(True)
        b.step(6)
        lone[1].step(6)
        assert np.array_equal(batched[1].get_populations(), lone[1].get_populations())


def test_autotune_on_d3q19_keeps_results():
    batched, lone = _pairs("spinodal3d", "fp32")
    with tl.TernaryBatch(batched) as b:
        variant, chunk = b.autotune(trial_steps=1)
        assert variant == 0  # one batched shape for periodic D3Q19
        n = batched[0].steps_done
        b.step(2)
        for e in lone:
            e.step(n + 2)
        for eb, el in zip(batched, lone):
            assert np.array_equal(eb.get_populations(), el.get_populations())


def test_sweep_members_batched_equal_lone_engines():
    """Members of the benchmark's 96-lattice contact-angle sweep (their own sizes,
    wells and wetting parameters from the library's inversion), batched under a
    graph at the autotuned tile, against the same lattices stepped alone."""
    members = W.sweep_wells(96)[:8]
    engines, lone = [], []
    for m in members:
        h = None
        for a in m["angles"]:
            try:
                h = tl.wetting_from_angles(m["kappa"], m["alpha"], *a)
                break
            except tl.TLBMError:
                continue
        rho, phi, psi = W.to_aux(*m["C"])
        for arr in (rho, phi, psi):
            arr[m["solid"] != 0] = 0.0
        for group in (engines, lone):
            e = tl.TernaryLB(9, m["nx"], m["ny"], 1, m["kappa"], m["alpha"], m["tau_f"], m["M_phi"], m["M_psi"],
                             h, m["solid"], "fp32")
            e.init_fields(rho, phi, psi)
            group.append(e)
    with tl.TernaryBatch(engines) as b:
        variant, chunk = b.autotune(trial_steps=1)
        b.set_graph(True)
        b.step(5)
        for e in lone:
            e.set_tile(variant, chunk)
            e.step(engines[0].steps_done)
        for eb, el in zip(engines, lone):
            assert np.array_equal(eb.get_populations(), el.get_populations())
            assert np.array_equal(eb.step_mass(), el.step_mass())
