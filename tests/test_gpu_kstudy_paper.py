"""The paper's study of the choice of k (Sec. 4.1 'Approximation Quality',
Fig. mseversusk, Table setups2D, Fig. effectsonapproximation), reproduced on
the GPU path in FP32 against the FP64 oracle.

Two problems shaped like Table setups2D:
* FWI: 251 x 251 grid over 0.02 m, N = 3200 steps of 7.5e-9 s, sine burst
  1 MHz, n_c = 2, psi0 = 1e12, homogeneous initial model (6000 m/s), four
  sources at the edge midpoints, receivers every 5th cell along the edges,
  homogeneous Neumann boundaries; the observed data come from a model with a
  slow inclusion, computed by the oracle on a grid twice as fine with twice
  the steps (the footnote of the study: no inverse crime);
* TATO: the density form on 363 x 363 over 9 m, N = 1800 steps of 3.4e-5 s,
  sine burst 650 Hz, psi0 = 1e2, air everywhere (gamma = 0), source at the
  left edge, pressure energy of a right-edge patch (Eq. cost2).
For each, k sweeps 22 decades around k0 = ||psi|| / ||f_adj|| (the automatic
rule at ratio 1).  The FP64 reference gradient g and the FP64 Algorithm 1
result at any k come from two oracle runs, at +k0 and -k0: K~(k) is affine in
k (Eq. superposedkernel1 on the discrete kernel: K~(k) = g + (k/2) K(l, l)),
so g is their mean and K(l, l) their difference over k0 (pinned on CPU).
The TATO problem is repeated with N = 1200, 4800 and 9600 and at a perturbed
design (the study's effect of N and of the design).

Asserted (the paper's qualitative findings): below some k the FP32 result
departs from FP64 and its error exceeds 100% (overflow/underflow: the head of
the hockey stick); at large k FP32 and FP64 agree and the error is the
neglected k^2 term, growing with k (the handle); between them a band of k
gives less than 5% error; the calibration rule of the study (decrease k until
FP32 and FP64 disagree, keep the smallest k before that) lands in the band;
N and the design shift the band only a little.  The measured table is printed.
"""
import numpy as np
import pytest
import torch

import oracle as O

from _oracle_pool import forward_traces, k0_of, pool, superposition_many

pytestmark = pytest.mark.gpu

EXPONENTS = list(range(-16, 7))   # k = k0 * 10^e: 23 values, 22 decades


@pytest.fixture(scope="module")
def W():
    import __graft_entry__ as ge
    ge.build()
    from paper_2509_15744_gb300 import wave
    return wave


def _edge_receivers(n, step=5):
    cells = set()
    for i in range(0, n, step):
        for (y, x) in ((0, i), (n - 1, i), (i, 0), (i, n - 1)):
            cells.add(y * n + x)
    return np.array(sorted(cells), np.int64)


def _fwi():
    n, L, N, dt, f, psi0, c0 = 251, 0.02, 3200, 7.5e-9, 1e6, 1e12, 6000.0
    h = L / (n - 1)
    init = np.full((n, n), c0)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    true = init.copy()
    true[(yy - 0.55 * n) ** 2 + (xx - 0.45 * n) ** 2 <= (0.15 * n) ** 2] = 0.5 * c0
    srcs = [(1, n // 2), (n - 2, n // 2), (n // 2, 1), (n // 2, n - 2)]
    rec = _edge_receivers(n)
    wav = O.sine_burst(np.arange(N + 1) * dt, f, 2, psi0)
    # observed data on the grid twice as fine with twice the steps: node i of
    # the coarse grid is node 2i, the model repeated, the Kronecker source x 2^2
    nf = 2 * n - 1
    tf = np.repeat(np.repeat(true, 2, axis=0), 2, axis=1)[:nf, :nf]
    wf = O.sine_burst(np.arange(2 * N + 1) * dt / 2, f, 2, 4.0 * psi0)
    recf = np.array([(r // n) * 2 * nf + (r % n) * 2 for r in rec], np.int64)
    spec_f = ("velocity", tf, h / 2, dt / 2, 2, "neumann")
    fine_jobs = [(spec_f, (2 * y) * nf + 2 * x, wf, recf, 2 * N) for (y, x) in srcs]
    shots = [(y * n + x, wav, rec, None, 1.0) for (y, x) in srcs]   # observed data filled in below
    return dict(name="FWI 251^2, N=3200", physics="velocity", param=init, h=h, dt=dt, N=N, bc="neumann",
                objective="l2", shots=shots, fine_jobs=fine_jobs)


def _tato(N=1800, design=None):
    n, L, dt, f, psi0 = 363, 9.0, 3.4e-5, 650.0, 1e2
    h = L / (n - 1)
    gamma = np.zeros((n, n)) if design is None else design
    y0, y1, x0 = (3 * n) // 8, (5 * n) // 8, n - n // 6
    py, px = np.meshgrid(np.arange(y0, y1), np.arange(x0, n), indexing="ij")
    patch = (py * n + px).ravel().astype(np.int64)
    wav = O.sine_burst(np.arange(N + 1) * dt, f, 2, psi0)
    shots = [((n // 2) * n + 2, wav, patch, None, O.patch_weight(len(patch), 1.0))]
    return dict(name=f"TATO 363^2, N={N}" + (", perturbed design" if design is not None else ""),
                physics="density", param=gamma, h=h, dt=dt, N=N, bc="neumann", objective="patch", shots=shots)


def _perturbed_design(n=363, seed=9):
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    d = gaussian_filter(rng.standard_normal((n, n)), 6.0)
    return np.clip(0.4 + d / (5 * d.std()), 0.0, 0.8)   # stays below the solid, within the time step's bound


def _spec(prob):
    return (prob["physics"], prob["param"], prob["h"], prob["dt"], 2, prob["bc"])


@pytest.fixture(scope="module")
def problems():
    """All oracle work of the study in one process pool: the FWI data on the
    fine grid, then k0 of every problem, then Algorithm 1 at +k0 and -k0."""
    probs = {"fwi": _fwi()}
    for N in (1200, 1800, 4800, 9600):
        probs[f"tato{N}"] = _tato(N)
    probs["tato_design"] = _tato(1800, _perturbed_design())
    with pool() as p:
        fine = p.map(forward_traces, probs["fwi"]["fine_jobs"])
        probs["fwi"]["shots"] = [(s, w, r, tr[:, ::2], wt)
                                 for (s, w, r, _, wt), tr in zip(probs["fwi"]["shots"], fine)]
        names = list(probs)
        k0s = p.map(k0_of, [(_spec(probs[n]), probs[n]["shots"][0], probs[n]["N"]) for n in names])
        jobs = []
        for n, k0 in zip(names, k0s):
            jobs += [(_spec(probs[n]), probs[n]["shots"], probs[n]["N"], k0),
                     (_spec(probs[n]), probs[n]["shots"], probs[n]["N"], -k0)]
        res = p.map(superposition_many, jobs, chunksize=1)
    for i, (n, k0) in enumerate(zip(names, k0s)):
        plus, minus = res[2 * i][0], res[2 * i + 1][0]
        probs[n]["k0"] = k0
        probs[n]["g"] = 0.5 * (plus + minus)      # the exact gradient
        probs[n]["B"] = (plus - minus) / k0       # K~(k) = g + (k/2) B
    return probs


def _gpu_side(W, prob, ks):
    dev = torch.device("cuda")
    m = W.Model(torch.from_numpy(prob["param"].astype(np.float32)).to(dev), prob["h"], prob["dt"], 2,
                prob["physics"], prob["bc"])
    shots = []
    for s, wav, rec, obs, _ in prob["shots"]:
        shots.append(W.Shot(s, torch.from_numpy(wav.astype(np.float32)).to(dev), torch.from_numpy(rec).to(dev),
                            None if obs is None else torch.from_numpy(obs.astype(np.float32)).to(dev)))
    out = []
    for k in ks:
        g, _, _ = m.gradient(shots, objective=prob["objective"], k=float(k))
        out.append(g.cpu().numpy().astype(np.float64))
    return out


def _study(W, prob):
    k0, g, B = prob["k0"], prob["g"], prob["B"]
    ks = [k0 * 10.0 ** e for e in EXPONENTS]
    gpu = _gpu_side(W, prob, ks)
    ng = np.linalg.norm(g)
    rows = []
    for e, k, kt in zip(EXPONENTS, ks, gpu):
        ref = g + 0.5 * k * B                               # FP64 Algorithm 1 at this k
        rows.append(dict(e=e, k=k, fp32=np.linalg.norm(kt - g) / ng, fp64=np.linalg.norm(ref - g) / ng,
                         diff=np.linalg.norm(kt - ref) / max(np.linalg.norm(ref), 1e-300)))
    print(f"\n{prob['name']}: k0 = {k0:.3e}")
    print("   log10(k/k0)   rel.err FP32   rel.err FP64   |FP32 - FP64|/|FP64|")
    for r in rows:
        print(f"   {r['e']:+4d}          {r['fp32']:.3e}      {r['fp64']:.3e}      {r['diff']:.3e}")
    return rows


def _band(rows, tol=0.05):
    """Width in decades of the range of k with FP32 error below tol, the
    crossings located by log-log interpolation between the sampled decades
    (0 if no sample is below tol)."""
    e = [r["e"] for r in rows]
    v = [np.log10(r["fp32"]) for r in rows]
    t = np.log10(tol)
    best = 0.0
    i = 0
    while i < len(rows):
        if v[i] >= t:
            i += 1
            continue
        j = i
        while j + 1 < len(rows) and v[j + 1] < t:
            j += 1
        lo = e[i] if i == 0 else e[i - 1] + (v[i - 1] - t) / (v[i - 1] - v[i]) * (e[i] - e[i - 1])
        hi = e[j] if j == len(rows) - 1 else e[j] + (t - v[j]) / (v[j + 1] - v[j]) * (e[j + 1] - e[j])
        best = max(best, hi - lo)
        i = j + 1
    return best


def _check_hockey_stick(rows, min_decades):
    # head: at the smallest k FP32 has lost the signal, FP64 has not
    assert rows[0]["fp32"] > 1.0 and rows[0]["fp64"] < 1e-6
    # handle: at the largest k the neglected k^2 term dominates; FP32 = FP64
    assert rows[-1]["fp64"] > 1.0 and abs(rows[-1]["fp32"] / rows[-1]["fp64"] - 1.0) < 0.1
    assert all(b["fp64"] > a["fp64"] for a, b in zip(rows, rows[1:]))
    # a band of k with less than 5% error
    assert _band(rows) >= min_decades
    # the calibration rule: from large k down, keep the smallest k before
    # FP32 and FP64 disagree (by more than 5%); that k lies in the band
    pick = None
    for r in reversed(rows):
        if r["diff"] > 0.05:
            break
        pick = r
    assert pick is not None and pick["fp32"] < 0.05


def test_fwi_k_study(W, problems):
    rows = _study(W, problems["fwi"])
    print(f"FWI band of k with < 5% error: {_band(rows):.2f} decades")
    _check_hockey_stick(rows, min_decades=1.5)


def test_tato_k_study_with_the_number_of_steps_and_the_design(W, problems):
    bands = {}
    best = {}
    for N in (1200, 1800, 4800, 9600):
        rows = _study(W, problems[f"tato{N}"])
        _check_hockey_stick(rows, min_decades=1.5)
        bands[N], best[N] = _band(rows), min(r["fp32"] for r in rows)
    rows = _study(W, problems["tato_design"])
    _check_hockey_stick(rows, min_decades=1.0)
    print(f"\nTATO bands of k with < 5% error (decades): { {n: round(b, 2) for n, b in bands.items()} }, "
          f"perturbed design: {_band(rows):.2f}")
    print(f"TATO best FP32 error per N: { {n: float(f'{b:.3e}') for n, b in best.items()} }, "
          f"perturbed design: {min(r['fp32'] for r in rows):.3e}")
    # more steps make the approximation somewhat worse, not unusable
    # (Fig. effectsonapproximation): the best error grows, the band narrows by
    # less than a decade
    assert best[9600] >= best[1200]
    assert bands[1200] - bands[9600] < 1.0
    assert _band(rows) >= bands[1800] - 1.5
