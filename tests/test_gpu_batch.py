"""Batched solver (lesbgk_batch_*): each slot gives, bitwise, what the same
problem gives alone through lesbgk_create/lesbgk_step, whatever else is in
the batch and whenever slots come and go; and a batch slot matches the FP64
oracle like the single-domain solver does."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1209_6548_gb300 import build as B
from paper_1209_6548_gb300 import inputs as I
from paper_1209_6548_gb300 import lesbgk as L
from tests.common import field_errors, oracle_params, record, rounding_bound, time_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def mixed_problems(nx=4, n=10, seed=3, with_q36=True):
    """The channel mix, a quarter on D2Q36, every third with Maxwell walls
    (specular share 0.3, Sec. 3.2), every fifth with heated walls (Sec. 4.2:
    T_w = wall_T + 0.02 sin(St t), St = pi sqrt(2)/8), and those k = 0, 5, 10,
    ... on D2Q16 with the D = 3 set D3Q64 instead."""
    probs = I.batch_mix(n=n, seed=seed, ny_lo=16, ny_hi=200)
    out = []
    for k, p in enumerate(probs):
        kw = dict(nx=nx)
        if with_q36 and k % 4 == 3:
            kw["nroots"] = 6
        if k % 3 == 1:
            kw["wall_specular"] = 0.3
        if k % 5 == 2:
            kw["wall_T_amp"] = 0.02
            kw["wall_T_freq"] = np.pi * np.sqrt(2.0) / 8.0
        if k % 5 == 0 and kw.get("nroots", p.nroots) == 4:
            kw["dim"] = 3
        from dataclasses import replace
        out.append(replace(p, **kw))
    return out


def alone(prob, steps):
    s = L.Solver(L.params_from_problem(prob))
    s.step(steps)
    return s.populations().cpu().numpy(), s.info.dt


def pool_for(probs, slack=2.0):
    return int(sum(L.batch_slot_bytes(L.params_from_problem(p)) for p in probs) * slack) + (1 << 20)


def test_batch_equals_alone_bitwise():
    probs = mixed_problems()
    bt = L.Batch(capacity=16, nx=4, pool_bytes=pool_for(probs))
    slots = [bt.add(L.params_from_problem(p)) for p in probs]
    steps = 64 * 2 + 7  # two graph replays and seven direct steps
    bt.step(steps)
    for p, sl in zip(probs, slots):
        ref, dt = alone(p, steps)
        got = bt.populations(sl).cpu().numpy()
        assert bt.info(sl).dt == dt
        assert bt.info(sl).steps_done == steps
        assert np.array_equal(got, ref), p.name


def test_slots_come_and_go():
    probs = mixed_problems(n=8, seed=5)
    bt = L.Batch(capacity=8, nx=4, pool_bytes=pool_for(probs))
    slots = [bt.add(L.params_from_problem(p)) for p in probs[:6]]
    bt.step(70)
    bt.remove(slots[2])
    bt.remove(slots[4])
    late = [bt.add(L.params_from_problem(p)) for p in probs[6:8]]
    bt.step(65)
    for i in (0, 1, 3, 5):
        ref, _ = alone(probs[i], 135)
        assert np.array_equal(bt.populations(slots[i]).cpu().numpy(), ref)
    for k, sl in enumerate(late):
        ref, _ = alone(probs[6 + k], 65)
        assert np.array_equal(bt.populations(sl).cpu().numpy(), ref)


def test_autotune_keeps_state_and_rows_do_not_change_bits():
    probs = mixed_problems(n=6, seed=7)
    bt = L.Batch(capacity=8, nx=4, pool_bytes=pool_for(probs))
    slots = [bt.add(L.params_from_problem(p)) for p in probs]
    bt.step(11)
    before = [bt.populations(s).cpu().numpy() for s in slots]
    chosen = bt.autotune((4, 16, 32, 64))
    assert chosen in (4, 16, 32, 64)
    for s, b0 in zip(slots, before):
        assert np.array_equal(bt.populations(s).cpu().numpy(), b0)
    bt.set_rows(5)
    bt.step(80)
    for p, s in zip(probs, slots):
        ref, _ = alone(p, 91)
        assert np.array_equal(bt.populations(s).cpu().numpy(), ref)


def test_residuals_decay_and_first_call_is_nan():
    prob = I.Problem(name="c", nx=4, ny=24, kn=0.2, b=-0.5, wall_ux=(-0.05, 0.05))
    bt = L.Batch(capacity=4, nx=4, pool_bytes=pool_for([prob]))
    s = bt.add(L.params_from_problem(prob))
    r0 = bt.residuals()
    assert np.isnan(r0).all()
    rs = []
    for _ in range(5):
        bt.step(200)
        rs.append(bt.residuals()[s])
    assert all(np.isfinite(rs)) and rs[-1] < rs[0] * 0.5


def test_pool_exhaustion_and_slot_limit():
    prob = I.Problem(name="c", nx=4, ny=100, kn=0.1, b=0.0)
    p = L.params_from_problem(prob)
    one = L.batch_slot_bytes(p)
    bt = L.Batch(capacity=8, nx=4, pool_bytes=3 * one + 100)
    got = [bt.try_add(p) for _ in range(5)]
    assert got[:3] == [0, 1, 2] and got[3] is None and got[4] is None
    bt.remove(1)
    assert bt.try_add(p) == 1
    small = L.Batch(capacity=2, nx=4, pool_bytes=10 * one)
    assert [small.try_add(p) for _ in range(3)][2] is None


@pytest.mark.parametrize("nx", [1, 2, 8, 32])
def test_other_widths(nx):
    probs = mixed_problems(nx=nx, n=5, seed=nx, with_q36=(nx != 32))
    bt = L.Batch(capacity=8, nx=nx, pool_bytes=pool_for(probs))
    slots = [bt.add(L.params_from_problem(p)) for p in probs]
    bt.step(66)
    for p, s in zip(probs, slots):
        ref, _ = alone(p, 66)
        assert np.array_equal(bt.populations(s).cpu().numpy(), ref)


def test_batch_slot_matches_oracle():
    prob = I.Problem(name="p", nx=4, ny=40, kn=0.1, b=0.5, g=(1e-3, 0.0), wall_T=(0.97, 1.02))
    bt = L.Batch(capacity=4, nx=4, pool_bytes=pool_for([prob]))
    s = bt.add(L.params_from_problem(prob))
    bt.step(300)
    dt = time_step(prob)
    op = oracle_params(prob, dt)
    f0 = O.init(op)
    f = O.run(op, f0, 300)
    ref, _ = O.moments(op, f)
    errs = field_errors(bt.moments(s).cpu().numpy(), ref, rounding_bound([f0, f], prob.nroots, prob.dim, 300,
                                                                         "f32", prob, dt))
    record("batch slot", errs)
    assert all(v["ok"] for v in errs.values()), errs


@pytest.mark.parametrize("spec", [0.0, 0.3])
def test_heated_slot_matches_oracle(spec):
    """Heated walls (Sec. 4.2) in a batch slot, admitted after the batch has
    stepped an odd number of times (its clock starts at its own admission),
    against the FP64 oracle within the derived bound."""
    from dataclasses import replace
    prob = replace(I.unsteady_heating(kn=0.1, amp=0.02, ny=40), wall_specular=spec)
    other = I.Problem(name="c", nx=4, ny=24, kn=0.2, b=-0.5, wall_ux=(-0.05, 0.05))
    bt = L.Batch(capacity=4, nx=4, pool_bytes=pool_for([prob, other]))
    bt.add(L.params_from_problem(other))
    bt.step(5)
    s = bt.add(L.params_from_problem(prob))
    bt.step(300)
    assert bt.info(s).steps_done == 300
    dt = time_step(prob)
    op = oracle_params(prob, dt)
    f0 = O.init(op)
    f = O.run(op, f0, 300)
    ref, _ = O.moments(op, f)
    errs = field_errors(bt.moments(s).cpu().numpy(), ref, rounding_bound([f0, f], prob.nroots, prob.dim, 300,
                                                                         "f32", prob, dt))
    record(f"batch heated spec {spec}", errs)
    assert all(v["ok"] for v in errs.values()), errs


@pytest.mark.parametrize("storage", [L.F16, L.BF16])
def test_16bit_slots_equal_alone_bitwise(storage):
    """FP16/BF16 slots beside FP32 ones (a class of their own per velocity set:
    one launch per class and step) give bitwise the populations of the
    single-domain solver in the same storage -- the stochastic rounding keyed
    by the instance's own step count and row -- through graph replays and
    direct steps, a slot admitted after an odd number of steps, heated walls,
    add_many and moments_many."""
    import torch
    probs = mixed_problems(n=10, seed=11)
    params = []
    for k, p in enumerate(probs):
        q = L.params_from_problem(p)
        if k % 2 == 0 and p.wall_specular == 0.0:  # (Maxwell walls take FP32 storage)
            q.storage = storage
        params.append(q)
    assert sum(q.storage == storage for q in params) >= 3
    assert any(q.storage == storage and q.wall_T_amp != 0.0 for q in params)
    bt = L.Batch(capacity=16, nx=4, pool_bytes=sum(L.batch_slot_bytes(q) for q in params) + (1 << 20))
    slots = bt.add_many(params[:-2])
    bt.step(7)
    late = [bt.add(q) for q in params[-2:]]  # admitted at buffer parity 1
    bt.step(64 * 2 + 5)
    for q, sl, n in zip(params, slots + late, [140] * (len(params) - 2) + [133, 133]):
        ref = L.Solver(q)
        ref.step(n)
        assert bt.info(sl).steps_done == n
        assert bool((bt.populations(sl) == ref.populations()).all()), (q.storage, q.ny)
        outs = [torch.empty((9, q.ny, q.nx), dtype=torch.float32, device="cuda")]
        bt.moments_many([sl], outs)
        assert bool((outs[0] == ref.moments()).all())
        ref.close()


def test_mismatched_nx_rejected():
    bt = L.Batch(capacity=2, nx=4, pool_bytes=1 << 20)
    with pytest.raises(L.LesbgkError):
        bt.add(L.make_params(nx=8, ny=16, kn=0.1, b=0.0))
    with pytest.raises(L.LesbgkError):
        bt.add(L.make_params(nx=4, ny=16, kn=0.1, b=0.0, nroots=4, order=4))
    with pytest.raises(L.LesbgkError):
        bt.add(L.make_params(nx=4, ny=16, kn=0.1, b=0.0, storage=L.F32C))
    with pytest.raises(L.LesbgkError):  # D3Q216 runs on its own three-warp kernel only
        bt.add(L.make_params(nx=4, ny=16, kn=0.1, b=0.0, nroots=6, order=4, dim=3))


def test_add_many_and_moments_many_match_the_per_slot_calls():
    """lesbgk_batch_add_many writes the same initial populations as one
    lesbgk_batch_add per solve (with and without initial fields), the solves
    step the same, and lesbgk_batch_moments_many returns the same fields as
    lesbgk_batch_moments, bitwise."""
    import torch
    probs = I.batch_mix(n=40, seed=3, ny_hi=128) + [I.Problem(name="q36", nroots=6, nx=4, ny=33, kn=0.1, b=0.5,
                                                             wall_ux=(-0.05, 0.05)),
                                                   I.unsteady_heating(kn=0.2, amp=0.02, ny=30),
                                                   I.Problem(name="d3", nx=4, ny=29, kn=0.1, b=-0.5, dim=3,
                                                             wall_ux=(-0.05, 0.05), wall_T=(0.98, 1.02))]
    params = [L.params_from_problem(p) for p in probs]
    # rough in y only: the mix runs the printed (unsplit) update, unstable for
    # fields that vary in x and y (the library's documented reading)
    inits = [np.repeat(I.random_fields(p, seed=k, amp_u=0.01, amp_T=0.01, amp_rho=0.01)[:, :, :1], p.nx, axis=2)
             if k % 3 == 0 else None for k, p in enumerate(probs)]
    pool = sum(L.batch_slot_bytes(p) for p in params) + (1 << 20)
    one = L.Batch(capacity=len(params), nx=4, pool_bytes=pool)
    many = L.Batch(capacity=len(params), nx=4, pool_bytes=pool)
    s1 = [one.add(p, h) for p, h in zip(params, inits)]
    s2 = many.add_many(params, inits)
    for a, b in zip(s1, s2):
        assert bool((one.populations(a) == many.populations(b)).all())
    one.step(70)
    many.step(70)
    outs = [torch.empty((9, p.ny, p.nx), dtype=torch.float32, device="cuda") for p in params]
    many.moments_many(s2, outs)
    for a, o in zip(s1, outs):
        assert bool((one.moments(a) == o).all())


def test_add_many_is_all_or_nothing():
    probs = I.batch_mix(n=6, seed=4, ny_hi=64)
    params = [L.params_from_problem(p) for p in probs]
    pool = sum(L.batch_slot_bytes(p) for p in params[:3])  # room for about half of them
    bt = L.Batch(capacity=6, nx=4, pool_bytes=pool)
    free0 = bt.pool_free()
    with pytest.raises(L.LesbgkError) as e:
        bt.add_many(params)
    assert e.value.code == L.ESPACE
    assert bt.pool_free() == free0 and not bt.params  # nothing kept
    assert len(bt.add_many(params[:3])) == 3


@pytest.mark.parametrize("k", [2, 16, 64])
def test_resident_kernel_is_bitwise_the_per_step_kernel(k):
    """Instances held in shared memory for k steps per launch give bitwise
    the populations of the per-step kernel, in a mix that straddles the
    shared-memory limit (some instances stay on the per-step path), through
    graph replays and single steps (an odd total: both buffer parities),
    with walls, force and both schemes."""
    from dataclasses import replace
    probs = I.batch_mix(n=16, seed=7, ny_lo=16, ny_hi=700)
    probs = [replace(p, scheme=I.SPLIT) if i % 2 else p for i, p in enumerate(probs)]
    params = [L.params_from_problem(p) for p in probs]
    pool = sum(L.batch_slot_bytes(p) for p in params) + (1 << 20)
    out = {}
    for on in (False, True):
        bt = L.Batch(capacity=len(params), nx=4, pool_bytes=pool)
        bt.set_resident(on, k, 1 << 20)  # every instance that fits
        slots = bt.add_many(params)
        bt.step(64 * 2 + 7)
        cfg = bt.launch()
        if on:
            assert cfg["resident"] and cfg["steps_per_launch"] == k and cfg["resident_max_ny"] >= 400
            assert any(p.ny <= cfg["resident_max_ny"] for p in probs) and any(p.ny > cfg["resident_max_ny"]
                                                                              for p in probs)
        out[on] = [bt.populations(s).cpu().numpy() for s in slots]
        bt.close()
    for a, b in zip(out[False], out[True]):
        assert np.array_equal(a, b)


def test_autotune_searches_rows_and_resident_modes():
    probs = I.batch_mix(n=32, seed=8, ny_hi=512)
    params = [L.params_from_problem(p) for p in probs]
    bt = L.Batch(capacity=len(params), nx=4, pool_bytes=sum(L.batch_slot_bytes(p) for p in params) + (1 << 20))
    slots = bt.add_many(params)
    bt.step(10)
    before = [bt.populations(s).cpu().numpy() for s in slots]
    rows = bt.autotune((8, 16, 32))
    cfg = bt.launch()
    assert cfg["rows_per_item"] == rows and rows in (8, 16, 32) and cfg["steps_per_launch"] in (16, 64)
    assert cfg["resident_max_ny"] in (64, 128, 256, 454) or not cfg["resident"]
    after = [bt.populations(s).cpu().numpy() for s in slots]
    assert all(np.array_equal(a, b) for a, b in zip(before, after))  # timing left the state alone


def test_guard_words_stay_intact_and_the_check_sees_a_change():
    """No batch kernel writes past its slot's memory: after admissions of every
    class (both sets, FP32/FP16/BF16, heated and Maxwell walls), steps through
    graphs, direct steps and the autotuner, removals and re-admissions, every
    slot's guard words are as admission left them; a guard overwritten on
    purpose is reported for that slot alone."""
    probs = mixed_problems(n=10, seed=21)
    params = []
    for k, p in enumerate(probs):
        q = L.params_from_problem(p)
        if k % 4 == 0 and p.wall_specular == 0.0:
            q.storage = L.F16 if k % 8 == 0 else L.BF16
        params.append(q)
    bt = L.Batch(capacity=12, nx=4, pool_bytes=sum(L.batch_slot_bytes(q) for q in params) + (1 << 20))
    slots = bt.add_many(params[:7])
    bt.step(64 + 3)
    bt.autotune((8, 16))
    bt.remove(slots[2])
    late = [bt.add(q) for q in params[7:]]
    bt.step(64 * 2 + 1)
    bt.moments_many([slots[0]], [__import__("torch").empty((9, params[0].ny, 4), device="cuda")])
    bad = bt.check_guards()
    assert not bad.any()
    bt.debug_poison(late[0])
    bad = bt.check_guards()
    assert bad[late[0]] == 1 and bad.sum() == 1


def test_checkpoint_and_resume_are_bitwise():
    """A slot's raw populations and step count (lesbgk_batch_get_raw), put into
    a fresh batch at another buffer parity (lesbgk_batch_set_raw), continue
    bitwise as the uninterrupted batch: FP32 and 16-bit slots, heated walls
    (their clock resumes with the step count) and Maxwell walls."""
    probs = mixed_problems(n=8, seed=31)
    params = []
    for k, p in enumerate(probs):
        q = L.params_from_problem(p)
        if k % 3 == 2 and p.wall_specular == 0.0:
            q.storage = L.F16 if k % 2 else L.BF16
        params.append(q)
    assert any(q.wall_T_amp != 0.0 for q in params) and any(q.storage != L.F32 for q in params)
    pool = sum(L.batch_slot_bytes(q) for q in params) + (1 << 20)
    a = L.Batch(capacity=8, nx=4, pool_bytes=pool)
    sa = a.add_many(params)
    a.step(64 + 9)
    cks = [a.checkpoint(s) for s in sa]
    a.step(64 * 2 + 5)
    b = L.Batch(capacity=10, nx=4, pool_bytes=pool)
    b.step(0)
    sb = b.add_many(params)
    b.step(1)  # another buffer parity than the checkpoint's batch
    for s, (raw, n) in zip(sb, cks):
        assert n == 64 + 9
        b.resume(s, raw, n)
    b.step(64 * 2 + 5)
    for x, y in zip(sa, sb):
        assert b.info(y).steps_done == a.info(x).steps_done
        assert bool((a.populations(x) == b.populations(y)).all())


def test_d3q64_slots_with_every_wall_model_equal_alone():
    """D3Q64 slots (the D = 3 set's z-even half) with heated, Maxwell, moving
    walls and a body force, in FP32 and 16-bit storage, admitted before and
    after an odd number of steps, equal their single-domain solves bitwise."""
    from dataclasses import replace
    base = I.Problem(name="d3", nx=4, ny=37, kn=0.1, b=-0.5, dim=3, wall_ux=(-0.05, 0.05), wall_T=(0.97, 1.03),
                     g=(1e-4, 0.0))
    probs = [replace(base, wall_T_amp=0.02, wall_T_freq=0.5553603672697958), replace(base, wall_specular=0.3),
             replace(base, ny=64, kn=0.05, b=0.5), replace(base, wall_T_amp=0.01, wall_T_freq=1.1, ny=20)]
    params = [L.params_from_problem(p) for p in probs]
    params[3].storage = L.F16
    params[2].storage = L.BF16
    bt = L.Batch(capacity=6, nx=4, pool_bytes=sum(L.batch_slot_bytes(q) for q in params) + (1 << 20))
    first = bt.add_many(params[:2])
    bt.step(9)
    late = [bt.add(q) for q in params[2:]]
    bt.step(64 + 11)
    for q, sl, n in zip(params, first + late, [84, 84, 75, 75]):
        ref = L.Solver(q)
        ref.step(n)
        assert bt.info(sl).steps_done == n and bt.info(sl).q == 32
        assert bool((bt.populations(sl) == ref.populations()).all()), (q.storage, q.wall_T_amp, q.wall_specular)
        ref.close()
