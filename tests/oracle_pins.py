"""Checks that pin the FP64 oracle to facts fixed outside itself.

Each check raises AssertionError on a mismatch. They are plain functions so
that ``test_oracle_pins.py`` runs them against the real oracle and
``test_oracle_mutants.py`` runs them against oracle builds with a planted
mistake (each mutant must fail at least one check).

Sources of truth:
  - hand traces derived on paper from §III.A-C (``golden/*.txt``);
  - closed forms of the update under a constant input (geometric series);
  - invariants stated in §III.A (weights positive, summing to one) and
    implied by the method (sorted rank keys, variance floor, |cpt| <= 3);
  - brute force: all permutations for the rank order (exact rational keys),
    exact rational prefix sums for B;
  - a special case that reduces to a library routine (scipy's binary
    opening for the 3x3 clean-up).
"""
from __future__ import annotations

import itertools
import os
import random
from fractions import Fraction

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _frac(s: str) -> float:
    return float(Fraction(s))


# ---------------------------------------------------------------- hand traces
def load_hand_trace(name="hand_trace_2x2.txt"):
    params, frames, outs, states, decs = {}, {}, {}, {}, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "param":
                params[tok[1]] = Fraction(tok[2])
            elif tok[0] == "frame":
                t = int(tok[1]); i = tok.index("depth")
                frames[t] = ([int(v) for v in tok[3:i]], [int(v) for v in tok[i + 1:]])
            elif tok[0] == "out":
                outs[(int(tok[1]), tok[2])] = [int(v) for v in tok[3:]]
            elif tok[0] == "state":
                states[(int(tok[1]), tok[2], tok[3])] = [_frac(v) for v in tok[4:]]
            elif tok[0] == "dec":
                decs[(int(tok[1]), int(tok[2]))] = [int(v) for v in tok[3:]]
    return params, frames, outs, states, decs


def check_hand_trace():
    params, frames, outs, states, decs = load_hand_trace()
    M = int(params["M"])
    g = O.OracleGMM(2, 2, M, float(params["alpha"]), float(params["k"]), float(params["T"]),
                    float(params["init_var"]), float(params["init_w"]),
                    v_min_c=float(params["v_min"]), v_min_d=float(params["v_min"]))
    for t in sorted(frames):
        grey, dep = frames[t]
        rgb = np.repeat(np.array(grey, np.uint8).reshape(2, 2, 1), 3, axis=2)
        out = g.tick(rgb, np.array(dep, np.uint16).reshape(2, 2), report=True)
        for p in range(4):
            exp = decs.get((t, p))
            if exp is not None:
                got = out["dec"].reshape(4, 6)[p].tolist()
                assert got == exp, f"frame {t} pixel {p} decisions: {got} != {exp}"
            # a stream without a step reports no margin
            assert (exp[0] == -2) == np.isinf(out["margin_c"].reshape(-1)[p])
            assert (exp[3] == -2) == np.isinf(out["margin_d"].reshape(-1)[p])
        for name in ("fg_rgb", "fg_d", "fused"):
            exp = outs.get((t, name))
            if exp is not None:
                got = out[name].reshape(-1).tolist()
                assert got == exp, f"frame {t} {name}: {got} != {exp}"
        exp = outs.get((t, "fusion_byte"))
        if exp is not None:
            got = g.fusion_bytes().reshape(-1).tolist()
            assert got == exp, f"frame {t} fusion byte: {got} != {exp}"
    for (p, stream, field), exp in states.items():
        if stream == "colour":
            got = {"w": g.wc[p], "mu": g.muc[p][:, 0], "v": g.vc[p]}[field]
            if field == "mu":  # grey input: all three channels equal
                assert np.array_equal(g.muc[p][:, 0], g.muc[p][:, 1])
                assert np.array_equal(g.muc[p][:, 0], g.muc[p][:, 2])
        else:
            got = {"w": g.wd[p], "mu": g.mud[p], "v": g.vd[p]}[field]
        assert np.allclose(got, exp, rtol=1e-7, atol=1e-12), f"pixel {p} {stream} {field}: {got} != {exp}"


def load_list1_traces(name="list1_traces.txt"):
    traces, cur = [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "trace":
                cur = {"name": tok[1], "F0": int(tok[2]), "steps": []}
            elif tok[0] == "step":
                cur["steps"].append((int(tok[1]), int(tok[2]), int(tok[4]), int(tok[5])))
            elif tok[0] == "end":
                traces.append(cur)
    return traces


def check_list1_traces():
    for tr in load_list1_traces():
        F, cpt = tr["F0"], 0
        for i, (r, d, eF, ec) in enumerate(tr["steps"]):
            F, cpt = O.fuse(r, d, F, cpt)
            assert (F, cpt) == (eF, ec), f"{tr['name']} step {i}: {(F, cpt)} != {(eF, ec)}"


def check_list1_properties(max_len=7):
    """Over every (rgb, d) sequence up to max_len from both labels: the
    counter stays in [-3, 3]; agreement sets the label to the common answer
    and clears the counter; on disagreement the label can change only on a
    step that starts with |cpt| = 3, and then it takes the answer of the
    stream the sign names (+3 colour, -3 depth)."""
    pairs = [(0, 0), (0, 1), (1, 0), (1, 1)]
    for F0 in (0, 1):
        for L in range(1, max_len + 1):
            for seq in itertools.product(range(4), repeat=L):
                F, cpt = F0, 0
                for s in seq:
                    r, d = pairs[s]
                    F1, c1 = O.fuse(r, d, F, cpt)
                    assert -3 <= c1 <= 3
                    if r == d:
                        assert (F1, c1) == (d, 0)
                    elif cpt == 3:
                        assert (F1, c1) == (r, 0)
                    elif cpt == -3:
                        assert (F1, c1) == (d, 0)
                    else:
                        assert F1 == F and abs(c1 - cpt) == 1
                    F, cpt = F1, c1


# ---------------------------------------------------------------- closed forms
def check_closed_form_constant_input(D=3, steps=200):
    """A component that matches a constant input c keeps matching, and
    mu_t = c + (mu_0 - c) r^t, v_t = r^t [v_0 + |mu_0 - c|^2 r (1 - r^t)],
    w_match(t) = 1 - (1 - w_0) r^t, w_other(t) = w_other(0) r^t, r = 1 - alpha
    (geometric series of the update; valid while v stays above v_min)."""
    alpha = 0.015625  # exact in float32
    r = 1.0 - alpha
    M = 4
    c = np.array([120.0, 64.0, 33.0][:D])
    mu0 = c + np.array([3.0, -2.0, 1.5][:D])
    v0 = 64.0
    e = float(np.sum((mu0 - c) ** 2))
    prm = O.stream_params(alpha, 2.5, 0.7, 900.0, 0.05, v_min=1e-3)
    w = np.array([0.55, 0.25, 0.15, 0.05])
    mu = np.zeros((M, D)); mu[0] = mu0
    for i in range(1, M):
        mu[i] = c + 500.0 + 40.0 * i
    v = np.array([v0, 400.0, 900.0, 1600.0])
    w_other0 = w[1:].copy()
    for t in range(1, steps + 1):
        fg, info = O.stream_step(prm, w, mu, v, c)
        assert info[0] == 0 and info[2] == 0 and fg == 0, f"t={t}: info {info}"
        rt = r ** t
        assert np.allclose(mu[0], c + (mu0 - c) * rt, rtol=1e-12, atol=1e-11)
        assert np.isclose(v[0], rt * (v0 + e * r * (1.0 - rt)), rtol=1e-11)
        assert np.isclose(w[0], 1.0 - (1.0 - 0.55) * rt, rtol=1e-12)
        assert np.allclose(w[1:], w_other0 * rt, rtol=1e-11)


def check_closed_form_depth():
    check_closed_form_constant_input(D=1, steps=150)


# ---------------------------------------------------------------- invariants
def check_invariants_random(seed=3, pixels=40, steps=120):
    rng = random.Random(seed)
    for p in range(pixels):
        M = 3 + p % 3
        D = 3 if p % 2 == 0 else 1
        alpha = rng.choice([0.01, 0.05, 0.2])
        v_min = rng.choice([1.0, 4.0])
        prm = O.stream_params(alpha, 2.5, rng.choice([0.5, 0.7, 0.9]), 225.0, 0.05, v_min=v_min)
        base = np.array([rng.uniform(20, 230) for _ in range(D)])
        w, mu, v = O.stream_init(M, D, 225.0, base)
        for t in range(steps):
            u = rng.random()
            if u < 0.7:
                x = base + np.array([rng.gauss(0, 3) for _ in range(D)])
            elif u < 0.85:
                x = base + 60.0
            else:
                x = np.array([rng.uniform(0, 255) for _ in range(D)])
            fg, info = O.stream_step(prm, w, mu, v, x)
            assert np.all(w > 0), w
            assert abs(w.sum() - 1.0) <= 1e-12, w.sum()
            assert np.all(v >= np.float32(v_min)), v
            key = w / np.sqrt(v)
            assert np.all(np.diff(key) <= 0), key
            j_before, B, rank_j, near = info
            assert 1 <= B <= M and 0 <= rank_j < M
            if j_before < 0:
                assert fg == 1
                assert np.array_equal(mu[rank_j], x) and v[rank_j] == np.float32(225.0)
            else:
                assert fg == int(rank_j >= B)


def check_special_case_T_near_one(seed=5):
    """T just below 1: the background set is every component, so any match
    is background."""
    rng = random.Random(seed)
    T = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    prm = O.stream_params(0.05, 2.5, T, 100.0, 0.3)
    for _ in range(20):
        w, mu, v = O.stream_init(5, 1, 100.0, [1000.0])
        for t in range(60):
            x = [1000.0 + (rng.gauss(0, 4) if rng.random() < 0.8 else rng.uniform(-800, 800))]
            fg, info = O.stream_step(prm, w, mu, v, x)
            if info[0] >= 0:
                assert fg == 0 and info[1] == 5, info


def check_first_match_wins():
    """Two components both within k sigma of the sample: the better ranked
    one (stored first) is the one that matches and gets updated (§III.A,
    test against the most weighted distribution first)."""
    prm = O.stream_params(0.25, 2.5, 0.7, 100.0, 0.05)
    w = np.array([0.5, 0.3, 0.2]); mu = np.array([[100.0], [104.0], [300.0]]); v = np.array([16.0, 16.0, 16.0])
    fg, info = O.stream_step(prm, w, mu, v, [103.0])
    assert info[0] == 0 and fg == 0
    assert np.isclose(mu[0, 0], 0.75 * 100.0 + 0.25 * 103.0) and mu[1, 0] == 104.0
    # strict threshold: d^2 == k^2 v exactly is not a match
    w = np.array([0.5, 0.3, 0.2]); mu = np.array([[100.0], [200.0], [300.0]]); v = np.array([16.0, 16.0, 16.0])
    fg, info = O.stream_step(prm, w, mu, v, [110.0])  # d^2 = 100 = 6.25 * 16
    assert info[0] == -1 and fg == 1
    # the bound is k standard deviations: d^2 = 79.21 lies between k v and k^2 v
    w = np.array([0.5, 0.3, 0.2]); mu = np.array([[100.0], [200.0], [300.0]]); v = np.array([16.0, 16.0, 16.0])
    fg, info = O.stream_step(prm, w, mu, v, [108.9])
    assert info[0] == 0 and fg == 0


# ---------------------------------------------------------------- brute force
def _brute_stable_rank(w, v):
    """Unique permutation with non-increasing key (compared exactly through
    w^2 / v as rationals) and equal keys in stored order."""
    M = len(w)
    k2 = [Fraction(w[i]) ** 2 / Fraction(v[i]) for i in range(M)]
    found = []
    for perm in itertools.permutations(range(M)):
        ok = True
        for a in range(M - 1):
            i, j = perm[a], perm[a + 1]
            if k2[i] < k2[j] or (k2[i] == k2[j] and i > j):
                ok = False
                break
        if ok:
            found.append(list(perm))
    assert len(found) == 1
    return found[0]


def check_rank_order_bruteforce():
    # every tie pattern: keys drawn from M levels, v in {1, 4, 16} so sqrt is exact
    for M in (3, 4, 5):
        levels = [Fraction(n, 64) for n in (3, 5, 7, 11, 13)][:M]
        vs = [1.0, 4.0, 16.0]
        for pat in itertools.product(range(M), repeat=M):
            v = np.array([vs[(i * 7 + pat[i]) % 3] for i in range(M)])
            w = np.array([float(levels[pat[i]]) * np.sqrt(v[i]) for i in range(M)])
            got = O.rank_order(w, v).tolist()
            exp = _brute_stable_rank(w, v)
            assert got == exp, f"pattern {pat}: {got} != {exp}"
    rng = random.Random(11)
    for _ in range(300):
        M = rng.choice([3, 4, 5])
        w = np.array([rng.uniform(0.01, 1.0) for _ in range(M)])
        v = np.array([rng.uniform(1.0, 400.0) for _ in range(M)])
        assert O.rank_order(w, v).tolist() == _brute_stable_rank(w, v)


def check_background_count_exact():
    # exact ties with dyadic weights: a prefix equal to T is not above it
    assert O.background_count(np.array([0.25, 0.25, 0.5]), 0.5) == 3
    assert O.background_count(np.array([0.5, 0.25, 0.25]), 0.5) == 2
    assert O.background_count(np.array([0.75, 0.125, 0.0625, 0.0625]), 0.75) == 2
    assert O.background_count(np.array([0.125, 0.125, 0.25, 0.5]), 0.999) == 4
    rng = random.Random(17)
    for _ in range(500):
        M = rng.choice([3, 4, 5])
        raw = [rng.randint(1, 1000) for _ in range(M)]
        tot = sum(raw)
        w = [Fraction(r, tot) for r in raw]
        T = Fraction(rng.randint(1, 999), 1000)
        # exact: first prefix strictly above T
        B = next((b + 1 for b in range(M) if sum(w[:b + 1]) > T), M)
        wf = np.array([float(x) for x in w])
        prefix = np.cumsum([float(x) for x in w])
        if np.any(np.abs(prefix - float(T)) < 1e-12):
            continue  # float rounding can legitimately decide an exact tie
        assert O.background_count(wf, float(T)) == B


def check_morph_open_against_scipy():
    import scipy.ndimage as ndi
    rng = np.random.default_rng(2)
    for H, W in ((1, 1), (1, 7), (5, 1), (9, 13), (32, 40)):
        for p in (0.3, 0.7, 0.95):
            m = (rng.random((H, W)) < p).astype(np.uint8)
            exp = ndi.binary_opening(m, structure=np.ones((3, 3)), border_value=0).astype(np.uint8)
            assert np.array_equal(O.morph_open3(m), exp)
    # a lone pixel vanishes, a 3x3 block away from the border survives
    m = np.zeros((7, 7), np.uint8); m[1, 1] = 1; m[3:6, 3:6] = 1
    out = O.morph_open3(m)
    assert out[1, 1] == 0 and out[3:6, 3:6].all() and out.sum() == 9


def check_depth_invalid_and_late_start():
    """Zero depth leaves the depth model untouched and copies the colour
    answer; the depth model starts at the first non-zero reading."""
    g = O.OracleGMM(1, 2, 3, 0.1, 2.5, 0.6, 100.0, 0.05)
    rgb = np.full((1, 2, 3), 90, np.uint8)
    g.tick(rgb, np.array([[0, 1200]], np.uint16))
    assert g.dinit.tolist() == [0, 1] and np.all(g.wd[0] == 0)
    rgb2 = rgb.copy(); rgb2[0, :, :] = 250  # colour miss everywhere
    out = g.tick(rgb2, np.array([[0, 1200]], np.uint16))
    assert out["fg_rgb"].tolist() == [[1, 1]]
    assert out["fg_d"].tolist() == [[1, 0]]   # invalid copies colour; valid matches
    assert np.all(g.wd[0] == 0) and g.dinit[0] == 0
    out = g.tick(rgb, np.array([[1500, 1200]], np.uint16))
    assert g.dinit[0] == 1 and out["fg_d"][0, 0] == 0
    assert np.allclose(g.mud[0], 1500.0) and np.allclose(g.wd[0], 1 / 3)


def check_closed_form_per_channel_variance():
    """With VAR_PER_CHANNEL the variance tracks |x - mu|^2 / D, so under a
    constant input v_t = r^t [v_0 + |mu_0 - c|^2 / D * r (1 - r^t)]."""
    alpha = 0.03125
    r = 1.0 - alpha
    for D, c, mu0 in ((3, np.array([80.0, 90.0, 100.0]), np.array([84.0, 87.0, 101.0])),
                      (1, np.array([1500.0]), np.array([1497.0]))):
        e = float(np.sum((mu0 - c) ** 2))
        prm = O.stream_params(alpha, 2.5, 0.7, 900.0, 0.05, v_min=1e-3,
                              flags=O.FLAG_VAR_PER_CHANNEL)
        w = np.array([0.7, 0.2, 0.1]); mu = np.zeros((3, D)); mu[0] = mu0
        mu[1] = c + 400.0; mu[2] = c + 900.0
        v = np.array([30.0, 500.0, 800.0])
        for t in range(1, 120):
            fg, info = O.stream_step(prm, w, mu, v, c)
            assert info[0] == 0 and info[2] == 0 and fg == 0
            rt = r ** t
            assert np.isclose(v[0], rt * (30.0 + e / D * r * (1.0 - rt)), rtol=1e-11), (D, t)
            assert np.allclose(mu[0], c + (mu0 - c) * rt, rtol=1e-12, atol=1e-10)


def check_rho_eta_against_scipy():
    """RHO_ETA: the matched component moves with rho = alpha * N(x; mu,
    sigma^2 I), the density taken from scipy, with sigma^2 = v / D by default
    and v under VAR_PER_CHANNEL."""
    from scipy.stats import multivariate_normal
    alpha = 0.25
    for D in (1, 3):
        for flags in (O.FLAG_RHO_ETA, O.FLAG_RHO_ETA | O.FLAG_VAR_PER_CHANNEL):
            mu0 = np.array([100.0, 50.0, 75.0][:D]); x = mu0 + np.array([1.5, -2.0, 0.5][:D])
            v0 = 6.0
            s2 = v0 if flags & O.FLAG_VAR_PER_CHANNEL else v0 / D
            rho = alpha * multivariate_normal.pdf(x, mean=mu0, cov=s2 * np.eye(D))
            prm = O.stream_params(alpha, 3.0, 0.7, 400.0, 0.05, v_min=1e-3, flags=flags)
            w = np.array([0.8, 0.15, 0.05]); mu = np.zeros((3, D)); mu[0] = mu0
            mu[1] = mu0 + 300.0; mu[2] = mu0 + 600.0
            v = np.array([v0, 400.0, 400.0])
            fg, info = O.stream_step(prm, w, mu, v, x)
            assert info[0] == 0 and info[2] == 0
            mu_new = (1 - rho) * mu0 + rho * x
            d2 = float(np.sum((x - mu_new) ** 2))
            if flags & O.FLAG_VAR_PER_CHANNEL:
                d2 /= D
            assert np.allclose(mu[0], mu_new, rtol=1e-13), (D, flags)
            assert np.isclose(v[0], (1 - rho) * v0 + rho * d2, rtol=1e-12), (D, flags)


def check_augmented_model():
    """The augmentation alternative: depth enters as a fourth channel scaled
    to the byte range; a zero reading takes the best-ranked component's depth
    mean, which is the same as feeding that value explicitly."""
    s = np.float32(255.0 / 4095.0)
    g = O.OracleAugmented(1, 2, 4, 0.05, 2.5, 0.7, 100.0, 0.05)
    rgb = np.array([[[90, 100, 110], [30, 40, 50]]], np.uint8)
    g.tick(rgb, np.array([[2000, 3000]], np.uint16))
    assert np.allclose(g.mu[0, :, 3], float(s) * 2000.0) and np.allclose(g.mu[1, :, 3], float(s) * 3000.0)
    # distinct components, in rank order, so that the imputed value is specific
    planes = g.planes()
    planes[:, 6, 0, 1] = [186.0, 170.0, 205.0, 150.0]   # depth-channel means
    planes[:, 0, 0, 1] = [0.55, 0.25, 0.15, 0.05]
    planes[:, 4, 0, 1] = [30.0, 60.0, 90.0, 120.0]
    g.set_state(planes)
    ref_w, ref_mu, ref_v = g.w[1].copy(), g.mu[1].copy(), g.v[1].copy()
    rgb2 = rgb.copy(); rgb2[0, 1] = (33, 38, 52)
    g.tick(rgb2, np.array([[2004, 0]], np.uint16))
    # the same step through the generic four-channel update with the imputed value
    prm = O.stream_params(0.05, 2.5, 0.7, 100.0, 0.05)
    x = np.array([33.0, 38.0, 52.0, ref_mu[0, 3]])
    O.stream_step(prm, ref_w, ref_mu, ref_v, x)
    assert np.array_equal(g.w[1], ref_w) and np.array_equal(g.mu[1], ref_mu)
    assert np.array_equal(g.v[1], ref_v)
    # Depth is one channel of four (§III.B, Fig. 2): with colour noise of
    # sigma 3 per channel the summed variance settles near 27, so a 150 mm
    # depth step at unchanged colour adds (150 s)^2 = 87 < k^2 v to the squared
    # distance and the augmented model misses it; the separate depth model
    # (sigma 5 mm) flags it.
    rng = np.random.default_rng(1)
    h = O.OracleAugmented(1, 1, 3, 0.05, 2.5, 0.7, 100.0, 0.05)
    sep = O.OracleGMM(1, 1, 3, 0.05, 2.5, 0.7, 100.0, 0.05)
    for t in range(80):
        c = np.clip(np.round(120 + rng.normal(0, 3, 3)), 0, 255).astype(np.uint8).reshape(1, 1, 3)
        d = np.array([[int(round(2500 + rng.normal(0, 5)))]], np.uint16)
        h.tick(c, d)
        sep.tick(c, d)
    c = np.full((1, 1, 3), 120, np.uint8)
    d = np.array([[2350]], np.uint16)
    assert h.tick(c, d)["fg"][0, 0] == 0
    assert sep.tick(c, d)["fg_d"][0, 0] == 1


# ---------------------------------------------------------------- F1 (Eq. 1-3)
def check_f1_hand_counted():
    """Confusion counts and Eq. 1-3 on a hand-counted 4x4 example (exact
    fractions), and the degenerate cases with empty denominators."""
    pred = truth = counts = scores = None
    cases = []
    with open(os.path.join(GOLDEN, "f1_confusion_4x4.txt")) as f:
        for line in f:
            tok = line.split()
            if not tok or tok[0].startswith("#"):
                continue
            if tok[0] == "pred":
                pred = np.array([int(v) for v in tok[1:]]).reshape(4, 4)
            elif tok[0] == "truth":
                truth = np.array([int(v) for v in tok[1:]]).reshape(4, 4)
            elif tok[0] == "counts":
                counts = [int(v) for v in tok[1:]]
            elif tok[0] == "scores":
                scores = [Fraction(v) for v in tok[1:]]
            elif tok[0] == "case":
                cases.append((np.array([int(c) for c in tok[3]]), np.array([int(c) for c in tok[5]]),
                              [int(v) for v in tok[7:11]], [Fraction(v) for v in tok[12:15]]))
    cases.insert(0, (pred, truth, counts, scores))
    for pr, tr, cnt, sc in cases:
        r = O.f1_scores(pr, tr)
        assert [r["tp"], r["fp"], r["fn"], r["tn"]] == cnt, (r, cnt)
        for name, want in zip(("recall", "precision", "f1"), sc):
            assert abs(r[name] - float(want)) <= 1e-15, (name, r[name], want)


# ---------------------------------------------------------------- near-threshold report
def _step_report(prm, w, mu, v, x):
    w = np.array(w, dtype=np.float64)
    mu = np.array(mu, dtype=np.float64).reshape(len(w), -1)
    v = np.array(v, dtype=np.float64)
    fg, info, margin = O.stream_step(prm, w, mu, v, x, with_margin=True)
    return info[0], info[3], margin


def check_near_threshold_report():
    """The near bits flag a decision within eps (relative) of its threshold
    and nothing farther, for each of the three decisions; the margin is that
    relative distance. Cases at (1 +- 5e-6) of a threshold must flag at
    eps = 1e-5 and cases at (1 +- 2e-5) must not, with every other decision
    of the step far from its threshold."""
    eps = 1e-5
    prm = O.stream_params(0.01, 2.5, 0.7, 16.0, 0.05, eps=eps)
    # Match: component 0 at mu 1000, v 16, k^2 v = 100; the others far away.
    for delta, near in ((-5e-6, True), (5e-6, True), (-2e-5, False), (2e-5, False)):
        x = 1000.0 + 10.0 * np.sqrt(1.0 + delta)
        j, bits, margin = _step_report(prm, [0.6, 0.3, 0.1], [1000.0, 5000.0, 9000.0],
                                       [16.0, 16.0, 16.0], [x])
        assert j == (0 if delta < 0 else -1), (delta, j)
        assert bits == (O.NEAR_MATCH if near else 0), (delta, bits)
        assert abs(margin - abs(delta)) <= 1e-9, (delta, margin)
    # Background set: the best component's updated weight at T (1 + delta).
    T = O.f32(0.7)
    for delta, near in ((-5e-6, True), (5e-6, True), (-2e-5, False), (2e-5, False)):
        w0 = (T * (1.0 + delta) - 0.01) / 0.99
        rest = 1.0 - w0
        j, bits, margin = _step_report(prm, [w0, 0.6 * rest, 0.4 * rest], [500.0, 800.0, 900.0],
                                       [16.0, 16.0, 16.0], [500.0])
        assert j == 0 and bits == (O.NEAR_T if near else 0), (delta, j, bits)
        assert abs(margin - abs(delta)) <= 1e-9, (delta, margin)
    # Sort keys: two unmatched components whose keys differ by a factor
    # (1 + delta) (both decay by the same factor, so the ratio stays).
    for delta, near in ((-5e-6, True), (5e-6, True), (-2e-5, False), (2e-5, False)):
        w1 = 0.2 * (1.0 + delta)
        j, bits, margin = _step_report(prm, [1.0 - w1 - 0.2, w1, 0.2], [500.0, 800.0, 900.0],
                                       [16.0, 16.0, 16.0], [500.0])
        want = abs(delta) / (1.0 + max(delta, 0.0))
        assert j == 0 and bits == (O.NEAR_KEY if near else 0), (delta, j, bits)
        assert abs(margin - want) <= 1e-9, (delta, margin)
    # Two components with the same w and v have the same key in any
    # arithmetic: a tie the stable order settles, not a near decision.
    j, bits, margin = _step_report(prm, [0.5, 0.25, 0.25], [500.0, 800.0, 900.0],
                                   [1.0, 4.0, 4.0], [500.0])
    assert j == 0 and bits == 0 and margin > 1e-2, (j, bits, margin)
    # Different parameters with exactly equal keys (w 1/4, v 4 and w 1/8,
    # v 1: both keys 1/8, and 1/16 after a dyadic update) are a tie only in
    # exact arithmetic: near, margin 0.
    prm2 = O.stream_params(0.5, 2.5, 0.7, 16.0, 0.05, eps=eps)
    j, bits, margin = _step_report(prm2, [0.625, 0.25, 0.125], [500.0, 800.0, 900.0],
                                   [1.0, 4.0, 1.0], [500.0])
    assert j == 0 and bits == O.NEAR_KEY and margin == 0.0, (j, bits, margin)
    # Same weight, variances 4 and 4 (1 + 4e-6): not twins, keys 2e-6 apart.
    j, bits, margin = _step_report(prm2, [0.5, 0.25, 0.25], [500.0, 800.0, 900.0],
                                   [1.0, 4.0, 4.0 * (1.0 + 4e-6)], [500.0])
    assert j == 0 and bits == O.NEAR_KEY and abs(margin - 2e-6) <= 1e-8, (j, bits, margin)


def check_near_threshold_boundary():
    """At exactly eps from a threshold the decision is flagged (the bound is
    inclusive). Dyadic values keep every step exact: eps = 1/64, alpha = 1/2,
    weights summing to one exactly."""
    eps = 1.0 / 64.0
    # Match: D = 3, k = 2, v = 16, so k^2 v = 64; x - mu = (8, 1, 0): d^2 = 65.
    prm = O.stream_params(0.5, 2.0, 0.7, 16.0, 0.05, eps=eps)
    j, bits, margin = _step_report(prm, [0.5, 0.3, 0.2],
                                   [[0.0, 0.0, 0.0], [200.0, 200.0, 200.0], [100.0, 100.0, 100.0]],
                                   [16.0, 16.0, 16.0], [8.0, 1.0, 0.0])
    assert j == -1 and bits == O.NEAR_MATCH and margin == eps, (j, bits, margin)
    # Background set: T = 3/4, updated best weight 0.5 * 67/128 + 0.5 = 195/256 = T (1 + eps).
    prm = O.stream_params(0.5, 2.0, 0.75, 16.0, 0.05, eps=eps)
    j, bits, margin = _step_report(prm, [67 / 128, 40 / 128, 21 / 128], [500.0, 800.0, 900.0],
                                   [1.0, 4.0, 16.0], [500.0])
    assert j == 0 and bits == O.NEAR_T and margin == eps, (j, bits, margin)
    # Keys: updated weights 1/8 (v = 1) and 63/256 (v = 4): keys 1/8 and 63/512,
    # apart by exactly eps times the larger.
    prm = O.stream_params(0.5, 2.0, 0.7, 16.0, 0.05, eps=eps)
    j, bits, margin = _step_report(prm, [0.2578125, 0.25, 0.4921875], [500.0, 800.0, 900.0],
                                   [1.0, 1.0, 4.0], [500.0])
    assert j == 0 and bits == O.NEAR_KEY and margin == eps, (j, bits, margin)


def check_near_bits_per_stream():
    """Image level: a near match in the depth stream lands in bits 4-6 and
    its margin in margin_d; the colour stream, far from every threshold,
    reports neither."""
    g = O.OracleGMM(1, 1, 3, 0.01, 2.5, 0.7, 16.0, 0.05)
    g.tick(np.full((1, 1, 3), 100, np.uint8), np.full((1, 1), 2000, np.uint16))
    planes = g.planes()
    planes[:, 0, 0, 0] = [0.6, 0.3, 0.1]          # colour weights
    planes[:, 5, 0, 0] = [0.6, 0.3, 0.1]          # depth weights
    planes[:, 1:4, 0, 0] = [[100.0] * 3, [180.0] * 3, [20.0] * 3]
    planes[:, 6, 0, 0] = [2000.0, 3000.0, 1000.0]
    v_d = 100.0 / (6.25 * (1.0 + 5e-6))             # d^2 = 100 = k^2 v_d (1 + 5e-6)
    planes[:, 7, 0, 0] = [v_d, 16.0, 16.0]
    planes[:, 4, 0, 0] = [16.0, 16.0, 16.0]
    g.set_state(planes, g.fusion_bytes())
    out = g.tick(np.full((1, 1, 3), 100, np.uint8), np.full((1, 1), 2010, np.uint16), report=True)
    assert out["near"][0, 0] == O.NEAR_MATCH << 4, out["near"]
    assert abs(out["margin_d"][0, 0] - 5e-6) <= 1e-9 and out["margin_c"][0, 0] > 1e-2, out
    # colour: matches component 0, weights (0.604, 0.297, 0.099) -> B = 2, rank 0;
    # depth: d^2 = 100 just above k^2 v, a miss; the replacement (weight
    # 0.05 / 0.941, v 16) ranks last, weights (0.631, 0.316, 0.053) -> B = 2
    assert out["dec"][0, 0].tolist() == [0, 2, 0, -1, 2, 2], out["dec"]


def check_margin_matches_near_bits(seed=9, pixels=60, steps=80):
    """Over random sequences, with eps large enough that near decisions
    occur: a step's near bits are set exactly when its margin is at most eps."""
    rng = np.random.default_rng(seed)
    eps = 0.02
    prm = O.stream_params(0.05, 2.5, 0.7, 50.0, 0.05, eps=eps)
    seen = [0, 0]
    for _ in range(pixels):
        w, mu, v = O.stream_init(4, 1, 50.0, [rng.uniform(0, 255)])
        base = rng.uniform(50, 200)
        for _ in range(steps):
            x = base + rng.normal(0, 6) + (rng.uniform(-80, 80) if rng.random() < 0.1 else 0.0)
            fg, info, margin = O.stream_step(prm, w, mu, v, [x], with_margin=True)
            assert (info[3] != 0) == (margin <= eps), (info, margin)
            seen[int(info[3] != 0)] += 1
    assert min(seen) > 20, seen


ALL_CHECKS = [
    check_hand_trace, check_list1_traces, check_list1_properties,
    check_closed_form_constant_input, check_closed_form_depth,
    check_invariants_random, check_special_case_T_near_one, check_first_match_wins,
    check_rank_order_bruteforce, check_background_count_exact,
    check_morph_open_against_scipy, check_depth_invalid_and_late_start,
    check_closed_form_per_channel_variance, check_rho_eta_against_scipy, check_augmented_model,
    check_f1_hand_counted, check_near_threshold_report, check_near_threshold_boundary,
    check_near_bits_per_stream, check_margin_matches_near_bits,
]
