"""Pins for oracle/surrogate.py (the learned radiance surrogate), against what the published methods
fix: trilinear interpolation reproduces affine fields and is continuous across cell faces (a
swapped weight or a wrong corner breaks both), the spatial hash's structure, back-propagation
against central finite differences in float64, Adam's closed form under a constant gradient and
its convergence on a quadratic, bfloat16 rounding against torch's conversion, and a training run
that fits a field."""
import numpy as np
import pytest

from oracle import surrogate as S

RES = (4, 6, 9, 13, 40, 64, 100, 150)     # levels 0-3 dense at T = 2^14, the rest hashed
SPEC = S.Spec(resolutions=RES, log2_table=14, aabb_lo=(-1.0, 0.0, -1.0), aabb_hi=(1.0, 2.0, 1.0))


def _points(n, seed, spec=SPEC, axis_normals=True):
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(spec.aabb_lo), np.asarray(spec.aabb_hi)
    pos = (lo[:, None] + (hi - lo)[:, None] * rng.uniform(0.02, 0.98, (3, n))).astype(np.float32)
    if axis_normals:
        nrm = np.zeros((3, n), np.float32)
        ax = rng.integers(0, 3, n)
        nrm[ax, np.arange(n)] = rng.choice([-1.0, 1.0], n)
    else:
        v = rng.normal(size=(3, n))
        nrm = (v / np.linalg.norm(v, axis=0)).astype(np.float32)
    return pos, nrm


def _params(spec, seed, scale_table=0.5):
    rng = np.random.default_rng(seed)
    L, T = spec.levels, spec.table_size
    table = rng.uniform(-scale_table, scale_table, (L, T, 2))
    w1 = rng.uniform(-1, 1, (S.HIDDEN, 2 * L)) * np.sqrt(6.0 / (2 * L + S.HIDDEN))
    w2 = rng.uniform(-1, 1, (S.HIDDEN, S.HIDDEN)) * np.sqrt(6.0 / (2 * S.HIDDEN))
    w3 = rng.uniform(-1, 1, (S.OUTPUTS, S.HIDDEN)) * np.sqrt(6.0 / (S.HIDDEN + S.OUTPUTS))
    return S.Params(table, w1, w2, w3)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-30, 30, 2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0, 3.4e38, 1e-40, -2.5]]).astype(np.float32)
    # exact ties: the 17th bit set, lower bits clear, both parities of the kept lsb
    ties = (np.array([0x3F808000, 0x3F818000, 0xC0108000], np.uint32)).view(np.float32)
    x = np.concatenate([x, ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(x), ref)


def test_direction_code_matches_cell_key_rule():
    n = np.array([[1, -1, 0, 0, 0, 0, 0.5, -0.0], [0, 0, 1, -1, 0, 0, 0.5, 0.0], [0, 0, 0, 0, 1, -1, 0.2, 0.0]],
                 np.float32)
    # ties go to x then y; the sign bit decides, so -0 counts as negative
    np.testing.assert_array_equal(S.direction_code(n), [0, 1, 2, 3, 4, 5, 0, 1])


def test_weights_partition_of_unity_and_corner_geometry():
    pos, nrm = _points(500, 2)
    idx, w = S.corners(SPEC, pos, nrm)
    np.testing.assert_allclose(w.sum(axis=2), 1.0, atol=1e-12)
    assert (w >= 0).all()
    # a point on a vertex (up to float32 rounding) puts all its weight on one corner
    R = RES[3]
    lo = np.asarray(SPEC.aabb_lo, np.float32)
    ext = np.asarray(SPEC.aabb_hi, np.float32) - lo
    v = np.array([[3], [5], [7]], np.float32)
    p = (lo[:, None] + ext[:, None] * v / np.float32(R)).astype(np.float32)
    _, wv = S.corners(SPEC, p, np.array([[0], [0], [1]], np.float32))
    assert abs(wv[0, 3].max() - 1.0) < 1e-5


def test_dense_addressing_is_injective_on_a_level():
    """Every vertex x direction of a dense level gets its own entry (brute force over the grid)."""
    R = RES[2]
    spec = SPEC
    lo = np.asarray(spec.aabb_lo, np.float64)
    ext = np.asarray(spec.aabb_hi, np.float64) - lo
    g = (np.arange(R) + 0.5) / R
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    seen = set()
    for d, nv in enumerate(([1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1])):
        pos = np.stack([lo[a] + ext[a] * c.reshape(-1) for a, c in enumerate((X, Y, Z))]).astype(np.float32)
        nrm = np.repeat(np.asarray(nv, np.float32)[:, None], pos.shape[1], axis=1)
        idx, _ = S.corners(spec, pos, nrm)
        seen |= set(idx[:, 2, :].reshape(-1).tolist())
    assert len(seen) == S.N_DIRS * (R + 1) ** 3
    assert max(seen) < spec.table_size


def test_hash_structure():
    """pi_x = 1 and XOR: along x with y, z, d fixed the hashed address is a bijection of x mod T;
    worked values of single-axis vertices."""
    spec = S.Spec(resolutions=(1 << 14,), log2_table=14, aabb_lo=(0, 0, 0), aabb_hi=(1, 1, 1))
    T = spec.table_size
    R = spec.resolutions[0]
    xs = (np.arange(R, dtype=np.float64) + 0.5) / R
    pos = np.stack([xs, np.full(R, 0.3), np.full(R, 0.7)]).astype(np.float32)
    nrm = np.repeat(np.array([[0], [1], [0]], np.float32), R, axis=1)
    idx, _ = S.corners(spec, pos, nrm)
    assert len(set(idx[:, 0, 0].tolist())) == T
    # vertex (0, 1, 0) of direction 0 hashes to 2654435761 = 0x9E3779B1 mod 2^14 = 0x39B1, (0, 0, 1)
    # to 805459861 = 0x30025795 mod 2^14 = 0x1795; direction 1 (normal -x) adds 2246822519 =
    # 0x85EBCA77 mod 2^14 = 0x0A77
    eps = np.float32(0.25 / R)
    p = np.array([[eps, eps, eps], [eps + 1.0 / R, eps, eps], [eps, eps, eps + 1.0 / R]], np.float32).T
    n = np.array([[1, 0, 0], [1, 0, 0], [-1, 0, 0]], np.float32).T
    idx, _ = S.corners(spec, p, n)
    assert idx[0, 0, 0] == 0 and idx[0, 0, 1] == 1
    assert idx[0, 0, 2] == 0x39B1 and idx[0, 0, 4] == 0x1795
    assert idx[1, 0, 0] == 1 and idx[1, 0, 1] == 2
    assert idx[2, 0, 0] == (0x0A77 ^ 0x1795)


def test_dense_level_reproduces_affine_fields():
    """Trilinear interpolation is exact on affine functions: fit a dense level's table to an affine
    field by least squares over many points, then the encoding reproduces it at new points."""
    spec = S.Spec(resolutions=(5,), log2_table=12, aabb_lo=(-1.0, 0.0, -1.0), aabb_hi=(1.0, 2.0, 1.0))
    a = np.array([0.3, -1.2, 0.7])
    b = np.array([-0.5, 0.25, 2.0])
    field = lambda p: (a @ p + 0.1, b @ p - 0.4)
    pos, _ = _points(4000, 3, spec)
    nrm = np.repeat(np.array([[0], [0], [1]], np.float32), pos.shape[1], axis=1)
    idx, w = S.corners(spec, pos, nrm)
    used = np.unique(idx[:, 0, :])
    col = {int(u): k for k, u in enumerate(used)}
    A = np.zeros((pos.shape[1], used.size))
    for c in range(8):
        A[np.arange(pos.shape[1]), [col[int(u)] for u in idx[:, 0, c]]] += w[:, 0, c]
    p64 = pos.astype(np.float64)
    table = np.zeros((1, spec.table_size, 2))
    for f in range(2):
        sol, *_ = np.linalg.lstsq(A, field(p64)[f], rcond=None)
        table[0, used, f] = sol
    pt, _ = _points(300, 4, spec)
    nt = np.repeat(np.array([[0], [0], [1]], np.float32), pt.shape[1], axis=1)
    e = S.encode(spec, table, pt, nt, emulate=False)
    ref = field(pt.astype(np.float64))
    np.testing.assert_allclose(e[:, 0], ref[0], atol=1e-6)
    np.testing.assert_allclose(e[:, 1], ref[1], atol=1e-6)


def test_encoding_is_continuous_across_cell_faces():
    """Any table: points just either side of a cell face encode to nearly the same features."""
    prm = _params(SPEC, 5)
    rng = np.random.default_rng(6)
    lo = np.asarray(SPEC.aabb_lo, np.float64)
    ext = np.asarray(SPEC.aabb_hi, np.float64) - lo
    for l, R in enumerate(RES):
        n = 64
        base = rng.uniform(0.1, 0.9, (3, n))
        ax = rng.integers(0, 3, n)
        face = np.round(base[ax, np.arange(n)] * R) / R
        h = 1e-6
        p0, p1 = base.copy(), base.copy()
        p0[ax, np.arange(n)] = face - h
        p1[ax, np.arange(n)] = face + h
        P0 = (lo[:, None] + ext[:, None] * p0).astype(np.float32)
        P1 = (lo[:, None] + ext[:, None] * p1).astype(np.float32)
        nrm = np.repeat(np.array([[0], [1], [0]], np.float32), n, axis=1)
        e0 = S.encode(SPEC, prm.table, P0, nrm, emulate=False)[:, 2 * l:2 * l + 2]
        e1 = S.encode(SPEC, prm.table, P1, nrm, emulate=False)[:, 2 * l:2 * l + 2]
        assert np.abs(e0 - e1).max() < 1e-3, l


def test_forward_closed_form_feature_selection():
    """W1 copies features 0..31 (and their negatives) into the hidden units, W2 is the identity,
    W3 sums units: y = sum of the level features' positive and negative parts = sum |e|."""
    L = SPEC.levels
    pos, nrm = _points(50, 7)
    prm = _params(SPEC, 8)
    w1 = np.zeros((64, 2 * L))
    w1[np.arange(2 * L), np.arange(2 * L)] = 1.0
    w1[2 * L + np.arange(2 * L), np.arange(2 * L)] = -1.0
    w3 = np.zeros((3, 64))
    w3[0, :] = 1.0
    w3[1, :2 * L] = 1.0
    w3[2, 2 * L:4 * L] = 1.0
    p = S.Params(prm.table, w1, np.eye(64), w3)
    e = S.encode(SPEC, prm.table, pos, nrm, emulate=False)
    y = S.forward(SPEC, p, pos, nrm, emulate=False)["y"]
    np.testing.assert_allclose(y[:, 0], np.abs(e).sum(axis=1), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(y[:, 1], np.maximum(e, 0).sum(axis=1), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(y[:, 2], np.maximum(-e, 0).sum(axis=1), rtol=1e-12, atol=1e-14)


def test_loss_worked_value():
    spec = SPEC
    y = np.array([[1.0, 0.0, 2.0]])
    t = np.array([[0.5, 0.1, 2.0]])
    # (0.25 / 1.01 + 0.01 / 0.01 + 0) / B, B = 2
    assert abs(S.loss(spec, y, t, np.ones(1), 2) - (0.25 / 1.01 + 1.0) / 2) < 1e-15


@pytest.mark.parametrize("emulate", [False])
def test_backward_matches_central_differences(emulate):
    """Every gradient (table entries, W1, W2, W3) against central differences of the loss with the
    denominator held at the unperturbed output (the no-gradient reading of the relative L2)."""
    spec = SPEC
    pos, nrm = _points(40, 9)
    prm = _params(spec, 10)
    rng = np.random.default_rng(11)
    target = rng.uniform(0, 2, (40, 3))
    mask = (rng.uniform(size=40) > 0.2).astype(np.float64)
    B = 48
    y0 = S.forward(spec, prm, pos, nrm, emulate)["y"]

    def L(p):
        return S.loss(spec, S.forward(spec, p, pos, nrm, emulate)["y"], target, mask, B, y_denominator=y0)

    L0, judge, g = S.backward(spec, prm, pos, nrm, target, mask, B, emulate)
    assert abs(L0 - L(prm)) < 1e-14
    np.testing.assert_allclose(judge[0], (mask[:, None] * np.abs(y0 - target)).sum(), rtol=1e-12)
    h = 1e-6
    checks = []
    idx, _ = S.corners(spec, pos, nrm)
    touched = [(l, int(idx[s, l, c]), f) for s in (0, 3, 17) for l in (0, 3, 5, 7) for c in (0, 5) for f in (0, 1)]
    for (l, i, f) in touched:
        pp, pm = prm.copy(), prm.copy()
        pp.table[l, i, f] += h
        pm.table[l, i, f] -= h
        checks.append(((L(pp) - L(pm)) / (2 * h), g.table[l, i, f]))
    for name, shape in (("w1", (64, 2 * spec.levels)), ("w2", (64, 64)), ("w3", (3, 64))):
        for k in range(12):
            i, j = rng.integers(0, shape[0]), rng.integers(0, shape[1])
            pp, pm = prm.copy(), prm.copy()
            getattr(pp, name)[i, j] += h
            getattr(pm, name)[i, j] -= h
            checks.append(((L(pp) - L(pm)) / (2 * h), getattr(g, name)[i, j]))
    fd = np.array([c[0] for c in checks])
    an = np.array([c[1] for c in checks])
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)
    assert np.abs(fd - an).max() <= 1e-6 * np.abs(an).max() + 1e-12
    # untouched table entries get no gradient
    mask_t = np.zeros(spec.table_size, bool)
    mask_t[idx[:, 1, :].reshape(-1)] = True
    assert (g.table[1][~mask_t] == 0).all()


def test_adam_closed_form_under_constant_gradient():
    """With a constant gradient g the bias-corrected moments are exactly g and g^2, so every step
    moves p by -lr g / (|g| + eps)."""
    spec = S.Spec(resolutions=(2,), log2_table=4, aabb_lo=(0, 0, 0), aabb_hi=(1, 1, 1), lr=0.01)
    rng = np.random.default_rng(12)
    prm = S.Params(rng.normal(size=(1, 16, 2)), rng.normal(size=(64, 2)), rng.normal(size=(64, 64)),
                   rng.normal(size=(3, 64)))
    g = S.Params(rng.normal(size=(1, 16, 2)), rng.normal(size=(64, 2)), np.zeros((64, 64)), rng.normal(size=(3, 64)))
    st = S.adam_init(prm)
    p = prm
    for t in range(1, 6):
        p = S.adam_step(spec, p, g, st)
        for name in ("table", "w1", "w2", "w3"):
            gg = getattr(g, name)
            ref = getattr(prm, name) - t * spec.lr * gg / (np.abs(gg) + spec.adam_eps)
            np.testing.assert_allclose(getattr(p, name), ref, rtol=1e-12, atol=1e-12)


def test_adam_converges_on_a_quadratic():
    spec = S.Spec(resolutions=(2,), log2_table=4, aabb_lo=(0, 0, 0), aabb_hi=(1, 1, 1), lr=0.05)
    c = np.random.default_rng(13).normal(size=(64, 64))
    p = S.Params(np.zeros((1, 16, 2)), np.zeros((64, 2)), np.zeros((64, 64)), np.zeros((3, 64)))
    st = S.adam_init(p)
    for _ in range(600):
        g = S.Params(np.zeros((1, 16, 2)), np.zeros((64, 2)), 2.0 * (p.w2 - c), np.zeros((3, 64)))
        p = S.adam_step(spec, p, g, st)
    assert np.abs(p.w2 - c).max() < 0.02


def test_training_fits_a_smooth_field():
    """Adam on the relative L2 fits a smooth radiance field over a few hundred steps: the loss drops
    by more than 20x and the held-out relative error falls below 5 %."""
    spec = S.Spec(resolutions=(4, 6, 9, 13), log2_table=12, aabb_lo=(-1.0, 0.0, -1.0), aabb_hi=(1.0, 2.0, 1.0),
                  lr=0.02)
    rng = np.random.default_rng(14)
    prm = _params(spec, 15, scale_table=1e-4)
    prm.w1 *= 3.0

    def field(pos):
        p = pos.astype(np.float64)
        base = 0.5 + 0.3 * np.sin(1.5 * p[0]) + 0.2 * p[1]
        return np.stack([base, 0.8 * base, 0.6 * base + 0.1 * p[2]], axis=1)

    st = S.adam_init(prm)
    first = None
    for it in range(300):
        pos, nrm = _points(256, 100 + it, spec)
        nrm[:] = np.array([[0], [1], [0]], np.float32)
        L, _, g = S.backward(spec, prm, pos, nrm, field(pos), emulate=False)
        first = L if first is None else first
        prm = S.adam_step(spec, prm, g, st)
    pos, nrm = _points(500, 7, spec)
    nrm[:] = np.array([[0], [1], [0]], np.float32)
    L_end, _, _ = S.backward(spec, prm, pos, nrm, field(pos), emulate=False)
    y = S.query(spec, prm, pos, nrm, emulate=False)
    rel = np.abs(y - field(pos)).sum() / np.abs(field(pos)).sum()
    assert L_end < first / 20
    assert rel < 0.05


def test_training_indices_are_pcg_draws():
    from oracle.hashing import pcg_hash
    idx = S.training_indices(7, 1000, 12345)
    seed = int(pcg_hash(8)[0])
    assert idx[0] == int(pcg_hash(0 ^ seed)[0]) % 12345
    assert idx[999] == int(pcg_hash(999 ^ seed)[0]) % 12345
    assert idx.min() >= 0 and idx.max() < 12345
    # roughly uniform: each tenth of the range gets 100 +- 40 draws
    h = np.bincount(idx * 10 // 12345, minlength=10)
    assert (np.abs(h - 100) < 40).all()


def test_emulated_precision_stays_near_float64():
    """The bfloat16 / float16 emulation moves outputs by about bfloat16's unit
    roundoff (2^-8) and gradients by a few times that (the relative loss divides by y^2 + eps)."""
    spec = SPEC
    pos, nrm = _points(256, 20)
    prm = _params(spec, 21)
    t = np.random.default_rng(22).uniform(0, 2, (256, 3))
    y64 = S.forward(spec, prm, pos, nrm, emulate=False)["y"]
    y16 = S.forward(spec, prm, pos, nrm, emulate=True)["y"]
    assert np.linalg.norm(y16 - y64) <= 2e-2 * np.linalg.norm(y64)
    _, _, g64 = S.backward(spec, prm, pos, nrm, t, emulate=False)
    _, _, g16 = S.backward(spec, prm, pos, nrm, t, emulate=True)
    for name in ("table", "w1", "w2", "w3"):
        a, b = getattr(g16, name), getattr(g64, name)
        assert np.linalg.norm(a - b) <= 0.1 * np.linalg.norm(b), name


def test_sparse_table_adam_leaves_untouched_entries_alone():
    """An entry with a zero gradient in a step keeps value and moments (so its later steps see the
    moments of its last touch), while a dense step would keep moving it by momentum."""
    spec = S.Spec(resolutions=(2,), log2_table=4, aabb_lo=(0, 0, 0), aabb_hi=(1, 1, 1), lr=0.01)
    rng = np.random.default_rng(30)
    prm = S.Params(rng.normal(size=(1, 16, 2)), rng.normal(size=(64, 2)), rng.normal(size=(64, 64)),
                   rng.normal(size=(3, 64)))
    g1 = S.Params(rng.normal(size=(1, 16, 2)), np.zeros((64, 2)), np.zeros((64, 64)), np.zeros((3, 64)))
    g2 = S.Params(g1.table.copy(), np.zeros((64, 2)), np.zeros((64, 64)), np.zeros((3, 64)))
    g2.table[0, :8] = 0.0   # entries 0..7 untouched in step 2
    g2.table[0, 8, 0] = 0.0  # entry 8: one feature zero, still touched
    st_s, st_d = S.adam_init(prm), S.adam_init(prm)
    ps = S.adam_step(spec, S.adam_step(spec, prm, g1, st_s), g2, st_s)
    pd = S.adam_step(spec, S.adam_step(spec, prm, g1, st_d, sparse_table=False), g2, st_d, sparse_table=False)
    after1 = S.adam_step(spec, prm, g1, S.adam_init(prm))
    np.testing.assert_array_equal(ps.table[0, :8], after1.table[0, :8])
    # entry 8 and beyond step in both forms alike; untouched entries drift only in the dense form
    np.testing.assert_allclose(ps.table[0, 8:], pd.table[0, 8:], rtol=0, atol=1e-15)
    assert np.all(np.abs(pd.table[0, :8] - after1.table[0, :8]) > 1e-4)
    np.testing.assert_array_equal(st_s.m.table[0, :8], (1 - spec.beta1) * g1.table[0, :8])
