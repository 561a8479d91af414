"""Pins of oracle.checkpointed: the gradient a checkpointing executor
computes when its checkpoints are stored in a lossy format (Sec. 3, Sec. 4).

Each pin compares it with something other than itself:
* the storage roundings, against closed-form float32 / binary16 / bfloat16
  cases (exact values, ties to even, overflow, subnormals, and the
  float32-first double rounding);
* identity storage, against the oracle's segment-regeneration gradient, bit
  for bit, for every number of slots (2D / 3D, OT2 / OT4);
* every state stored (M = N), against the imaging condition written out
  from the decoded states n <= N-2 and the live state N-1;
* a schedule traced by hand (N = 5, M = 2), which recomputes a state from a
  decoded checkpoint;
* the error's dependence on the storage precision.
"""
import numpy as np
import pytest

from oracle import checkpointed as K
from oracle import propagator as O
from oracle import revolve as R

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rt(x, store):
    return K.roundtrip(np.asarray(x, dtype=np.float64), store)


# ---------------------------------------------------------------- roundings

def test_fp32_rounding_ties_to_even():
    one = 1.0
    assert _rt([one + 2.0 ** -24], "fp32")[0] == one                    # tie, even below
    assert _rt([one + 3 * 2.0 ** -24], "fp32")[0] == one + 2.0 ** -22   # tie, even above
    assert _rt([one + 2.0 ** -24 + 2.0 ** -40], "fp32")[0] == one + 2.0 ** -23


def test_fp16_rounding_closed_form_cases():
    vals = np.array([1.0, -2.5, 1024.0, 65504.0, 2.0 ** -14, 2.0 ** -24])   # representable
    assert np.array_equal(_rt(vals, "fp16"), vals)
    assert _rt([1 + 2.0 ** -11], "fp16")[0] == 1.0                     # tie, even below
    assert _rt([1 + 3 * 2.0 ** -11], "fp16")[0] == 1 + 2.0 ** -9       # tie, even above
    assert _rt([1 + 2.0 ** -11 + 2.0 ** -20], "fp16")[0] == 1 + 2.0 ** -10
    assert _rt([2.0 ** -25], "fp16")[0] == 0.0                         # subnormal tie to 0
    assert _rt([3 * 2.0 ** -25], "fp16")[0] == 2.0 ** -23              # subnormal tie, even above
    assert _rt([65519.0], "fp16")[0] == 65504.0
    with pytest.raises(ValueError):
        _rt([65520.0], "fp16")                                          # rounds to infinity
    # the decision is taken on the float32 value: 1 + 2^-11 + 2^-40 is above
    # the binary16 tie in FP64, but its float32 value is the tie itself
    assert _rt([1 + 2.0 ** -11 + 2.0 ** -40], "fp16")[0] == 1.0


def test_bf16_rounding_closed_form_cases():
    vals = np.array([1.0, -2.5, 3.140625, 2.0 ** 100, 2.0 ** -126])
    assert np.array_equal(_rt(vals, "bf16"), vals)
    assert _rt([1 + 2.0 ** -8], "bf16")[0] == 1.0                      # tie, even below
    assert _rt([1 + 3 * 2.0 ** -8], "bf16")[0] == 1 + 2.0 ** -6        # tie, even above
    assert _rt([1 + 2.0 ** -8 + 2.0 ** -20], "bf16")[0] == 1 + 2.0 ** -7
    assert _rt([-(1 + 3 * 2.0 ** -8)], "bf16")[0] == -(1 + 2.0 ** -6)  # sign-symmetric
    big = float(np.finfo(np.float32).max)
    with pytest.raises(ValueError):
        _rt([big], "bf16")                                              # rounds to infinity
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4096) * 10.0 ** rng.uniform(-20, 20, 4096)
    y = _rt(x, "bf16")
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(y - x32) <= 2.0 ** -8 * np.abs(x32))           # half an ulp of 8 bits
    assert np.all((y.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_codec_storage_keeps_its_bound():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((13, 17, 9)) * 0.3
    tol = 1e-3
    y = K.roundtrip(x, "codec", tol=tol)
    assert np.max(np.abs(y - x.astype(np.float32))) <= tol
    z = K.roundtrip(x, "rate", rate=32)
    assert np.max(np.abs(z - x.astype(np.float32))) < 1e-5


# ---------------------------------------------------------------- executor

def _case(dims, so, time_order, nt, seed=2):
    if dims == 2:
        shape, nbl = (41, 53), 8
        src = (20.0, 0.0, 150.0)
        rec = np.array([[15.0, 0.0, 30.0 + 20.0 * i] for i in range(12)])
    else:
        shape, nbl = (19, 21, 23), 4
        src = (20.0, 60.0, 70.0)
        rec = np.array([[15.0, 40.0 + 10.0 * (i % 3), 30.0 + 20.0 * (i // 3)] for i in range(9)])
    g = O.Grid(dims=dims, shape=shape, nbl=nbl, h=10.0, so=so, dt=0.8 if so > 4 else 1.0, nt=nt,
               vmax_damp=3.0, time_order=time_order)
    rng = np.random.default_rng(seed)
    vel = 2.0 + 0.5 * rng.random(shape)
    ser = O.ricker(nt, g.dt, 0.025, 30.0)
    dobs = O.forward(g, vel * 1.03, [src], ser, rec)
    return g, vel, [src], ser, rec, dobs


@pytest.mark.parametrize("dims,so,time_order,nt", [(2, 4, 2, 60), (2, 8, 4, 50), (3, 4, 2, 40), (3, 4, 4, 30)])
def test_identity_storage_is_the_segment_gradient_bitwise(dims, so, time_order, nt):
    g, vel, src, ser, rec, dobs = _case(dims, so, time_order, nt)
    phi0, g0, _ = O.gradient(g, vel, src, ser, rec, dobs)
    for M in (2, 3, 7, nt - 1, nt):
        phi, gr, cnt = K.gradient(g, vel, src, ser, rec, dobs, M, store="fp64")
        assert np.array_equal(gr, g0), M
        assert abs(phi - phi0) <= 1e-13 * phi0
        assert cnt["p"] == R.p_closed(nt, M)


def _explicit_gradient(g, vel, src, ser, rec, r, states):
    """sum_n lam^n (A u~^n + q^n) c^2 (+ dt^2/12 c^4 lap u~^n lap lam^n for
    OT4), with lam^n from the adjoint recursion and u~^n = states[n]."""
    N = g.nt
    c2 = vel * vel
    idx, wt = O.interp(g, np.asarray(src[0], dtype=np.float64))
    lam = {}
    with K.Stepper(g, vel, src, ser, rec) as S:
        l1 = l2 = np.zeros(g.shape)
        for j in range(N, 0, -1):
            l0 = S.adj(r, j, l1, l2)
            lam[j - 1] = l0
            l1, l2 = l0, l1
    grad = np.zeros(g.shape)
    k = g.dt * g.dt / 12.0
    for n in range(N - 1, -1, -1):
        u = states[n]
        Au = O.laplacian(g, u)
        if g.time_order == 4:
            Au = Au + k * O.laplacian(g, c2 * O.laplacian(g, u))
        q = np.zeros(g.shape)
        np.add.at(q.reshape(-1), idx, wt * ser[n])
        grad += lam[n] * (Au + q) * c2
        if g.time_order == 4:
            grad += k * c2 * c2 * O.laplacian(g, u) * O.laplacian(g, lam[n])
    return grad


def _trajectory(g, vel, src, ser, rec):
    us = [np.zeros(g.shape)]
    prev = np.zeros(g.shape)
    with K.Stepper(g, vel, src, ser, rec) as S:
        for n in range(g.nt - 1):
            nxt = S.fwd(n, us[-1], prev)
            prev = us[-1]
            us.append(nxt)
    return us


def _residual(g, vel, src, ser, rec, dobs):
    d = O.forward(g, vel, src, ser, rec)
    r = np.ascontiguousarray(d - dobs)
    r[0] = 0.0
    return r


@pytest.mark.parametrize("time_order", [2, 4])
@pytest.mark.parametrize("store,kw", [("fp16", {}), ("codec", {"tol": 5e-3}), ("rate", {"rate": 10})])
def test_every_state_stored_reads_the_decoded_states(time_order, store, kw):
    # M = N: the first sweep stores states 1..N-1, reverses N-1 from the
    # live state, then restores every state n <= N-2 right before its turn
    nt = 24
    g, vel, src, ser, rec, dobs = _case(2, 4, time_order, nt)
    acts, _ = R.schedule(nt, nt)
    turns = [a for op, a, _ in acts if op == R.YOUTURN]
    assert turns == list(range(nt - 1, -1, -1))
    us = _trajectory(g, vel, src, ser, rec)
    states = {n: K.roundtrip(us[n], store, **kw) for n in range(1, nt - 1)}
    states[0] = np.zeros(g.shape)
    states[nt - 1] = us[nt - 1]
    r = _residual(g, vel, src, ser, rec, dobs)
    expect = _explicit_gradient(g, vel, src, ser, rec, r, states)
    _, got, _ = K.gradient(g, vel, src, ser, rec, dobs, nt, store=store, **kw)
    assert np.max(np.abs(got - expect)) <= 1e-12 * np.max(np.abs(expect))
    _, exact, _ = O.gradient(g, vel, src, ser, rec, dobs)
    assert np.max(np.abs(got - exact)) > 1e-6 * np.max(np.abs(exact))   # the storage is visible


@pytest.mark.parametrize("store,kw", [("fp16", {}), ("bf16", {}), ("codec", {"tol": 1e-2})])
def test_hand_traced_schedule_recomputes_from_the_decoded_checkpoint(store, kw):
    # N = 5, M = 2: advance 0->2, store (u2, u1) in slot 1, advance 2->4,
    # turn 4 (live); restore slot 1, advance 2->3, turn 3 (recomputed from
    # the decoded pair); restore slot 1, turn 2 (decoded); restore slot 0,
    # advance 0->1, store (u1, u0) in slot 1, turn 1 (live, recomputed from
    # the exact zero state); restore slot 0, turn 0 (zero state)
    A, T, S_, Y = R.ADVANCE, R.TAKESHOT, R.RESTORE, R.YOUTURN
    acts, _ = R.schedule(5, 2)
    assert acts == [(A, 0, 2), (T, 2, 1), (A, 2, 2), (Y, 4, 0), (S_, 2, 1), (A, 2, 1), (Y, 3, 0),
                    (S_, 2, 1), (Y, 2, 0), (S_, 0, 0), (A, 0, 1), (T, 1, 1), (Y, 1, 0), (S_, 0, 0),
                    (Y, 0, 0)]
    g = O.Grid(dims=2, shape=(24, 28), nbl=4, h=10.0, so=4, dt=1.0, nt=5, vmax_damp=3.0)
    rng = np.random.default_rng(7)
    vel = 2.0 + 0.3 * rng.random(g.shape)
    src = [(70.0, 0.0, 90.0)]
    ser = np.array([1.0, -0.7, 0.45, 0.2, -0.1])
    rec = np.array([[40.0, 0.0, 20.0 + 15.0 * i] for i in range(8)])
    dobs = O.forward(g, vel * 1.05, src, ser, rec)
    r = _residual(g, vel, src, ser, rec, dobs)
    E = lambda x: K.roundtrip(x, store, **kw)
    z = np.zeros(g.shape)
    with K.Stepper(g, vel, src, ser, rec) as S:
        u1 = S.fwd(0, z, z)
        u2 = S.fwd(1, u1, z)
        u3 = S.fwd(2, u2, u1)
        u4 = S.fwd(3, u3, u2)
        states = {4: u4, 3: S.fwd(2, E(u2), E(u1)), 2: E(u2), 1: u1, 0: z}
        expect = np.zeros(g.shape)
        l1 = l2 = z
        for j in range(5, 0, -1):
            l0 = S.adj(r, j, l1, l2, un=states[j - 1], grad=expect)
            l1, l2 = l0, l1
    _, got, _ = K.gradient(g, vel, src, ser, rec, dobs, 2, store=store, **kw)
    assert np.array_equal(got, expect)
    _, exact, _ = O.gradient(g, vel, src, ser, rec, dobs)
    assert not np.array_equal(got, exact)


def test_error_follows_the_storage_precision():
    g, vel, src, ser, rec, dobs = _case(2, 4, 2, 60)
    _, exact, _ = O.gradient(g, vel, src, ser, rec, dobs)

    def err(store, **kw):
        _, gr, _ = K.gradient(g, vel, src, ser, rec, dobs, 4, store=store, **kw)
        return np.linalg.norm(gr - exact) / np.linalg.norm(exact)

    # rounding errors scale with the unit roundoff: 2^-24, 2^-11, 2^-8
    e32, e16, eb = err("fp32"), err("fp16"), err("bf16")
    assert 2.0 ** -16 / 4 < e32 / eb < 2.0 ** -16 * 4
    assert 8.0 / 3 < eb / e16 < 8.0 * 3
    _, u = O.forward(g, vel, src, ser, rec, want_final=True)
    umax = float(np.abs(u).max())
    ec = [err("codec", tol=t * umax) for t in (1e-2, 1e-3, 1e-4)]
    assert ec[0] > ec[1] > ec[2]
    er = [err("rate", rate=b) for b in (8, 12, 16)]
    assert er[0] > er[1] > er[2]


def test_step_interface_rejects_bad_calls():
    g, vel, src, ser, rec, dobs = _case(2, 4, 2, 8)
    z = np.zeros(g.shape)
    r = np.zeros((g.nt + 1, len(rec)))
    with K.Stepper(g, vel, src, ser, rec) as S:
        for n in (-1, g.nt):
            with pytest.raises(ValueError):
                S.fwd(n, z, z)
        for j in (0, g.nt + 1):
            with pytest.raises(ValueError):
                S.adj(r, j, z, z)
        with pytest.raises(ValueError):
            S.adj(r, 1, z, z, un=None, grad=np.zeros(g.shape))   # a gradient needs u^{j-1}
    with pytest.raises(ValueError):
        K.Stepper(g, vel[:-1], src, ser, rec)
    with pytest.raises(ValueError):
        K.gradient(g, vel, src, ser, rec, dobs, 2, store="fp8")
    with pytest.raises(ValueError):
        K.gradient(g, vel, src, ser, rec, dobs, 2, store="codec")        # no tolerance
