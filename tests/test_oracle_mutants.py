"""The oracle's pins catch plausible mistakes: each case below plants one
mistake in the oracle's source (a flipped sign, a dropped term, an operand
used in the wrong place, an off-by-one rank, a wrong tie-break or stopping
rule, a permutation used in the wrong direction), on the CPU only, and the
pin files must then fail.

No copy of the oracle is made: the runner below (this file run as a script)
reads one oracle module's source, applies the replacement, executes it as
that module in ``sys.modules`` and runs the pin files with pytest in the same
process.  Each case runs in its own subprocess; several run at once.

The one plausible change not caught is folding the second projection pass's
coefficients into the core (Brand's update: P = U^T D after two passes).
Those coefficients are U^T (D - U U^T D), zero in exact arithmetic; the pass
removes rounding only, so no pin above rounding level can see it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_fastpi.py", "tests/test_oracle_reorder.py"]

# (module, original text, planted mistake, description); the original text
# occurs exactly once in the module.
MUTANTS = [
    ("fastpi", "R = D - Uc @ P\n", "R = D + Uc @ P\n", "residual: wrong sign of the projection"),
    ("fastpi", "K[:k, k:] = P\n", "K[:k, k:] = -P\n", "core: wrong sign of the projection block"),
    ("fastpi", "K[:k, k:] = P\n", "K[:k, k:] = 0\n", "core: projection block dropped"),
    ("fastpi", "K[:k, :k] = np.diag(sig)\n", "K[:k, :k] = np.eye(k)\n", "core: Sigma dropped"),
    ("fastpi", "Wnew[q:] = Vk[k:]\n", "Wnew[q:] = 0\n", "coefficients of the appended columns dropped"),
    ("fastpi", "Unew = np.hstack([Uc, Q]) @ Uk[:, :kk]\n", "Unew = np.hstack([Uc, Q])[:, :kk]\n",
     "left basis not rotated by the core's singular vectors"),
    ("fastpi", "RR[:, piv] = RRp[:rank]\n", "RR[:, :] = RRp[:rank]\n", "column pivoting not undone"),
    ("fastpi", "rank = int(np.count_nonzero(d > drop_tol * dmax)) if dmax > 0 else 0\n",
     "rank = int(d.size)\n", "dependent residual directions kept"),
    ("fastpi", "return (r * np.asarray(x, dtype=np.int64) + n - 1) // n",
     "return (r * np.asarray(x, dtype=np.int64)) // n", "floor(alpha x) instead of ceil"),
    ("fastpi", "s_i = np.minimum(np.minimum(ceil_alpha(ni, r, n), mi), ni)",
     "s_i = np.minimum(np.minimum(ceil_alpha(mi, r, n), mi), ni)", "block rank from m_1i instead of n_1i"),
    ("fastpi", "s = int(min(ceil_alpha(n1, r, n), S + m2, n1))", "s = int(min(ceil_alpha(n1, r, n), S + m2))",
     "row-phase rank not capped by n1"),
    ("fastpi", "rr = int(min(r, m, s + n2))", "rr = int(min(r, m, s + n2 + 1))", "column-phase rank off by one"),
    ("fastpi", "Urow = np.vstack([U1 @ W[:S], W[S:]])", "Urow = np.vstack([U1 @ W[:S], -W[S:]])",
     "row phase: wrong sign on the A21 rows of U"),
    ("fastpi", "V = np.vstack([Vrow @ W[:s], W[s:]])", "V = np.vstack([Vrow @ W[:s], 0 * W[s:]])",
     "column phase: T rows of V dropped"),
    ("fastpi", "M = np.vstack([sig1[:, None] * V1.T, A21.toarray()])", "M = np.vstack([V1.T, A21.toarray()])",
     "Eq. 2 single shot: Sigma1 dropped"),
    ("fastpi", "N = np.hstack([Urow * sig_row[None, :], T.toarray()])", "N = np.hstack([Urow, T.toarray()])",
     "Eq. 3 single shot: Sigma_row dropped"),
    ("fastpi", "return max(m, n) * EPS * float(np.max(S))", "return 0.5 * float(np.max(S))",
     "pseudoinverse threshold too large"),
    ("fastpi", "return fac.V @ (inv[:, None] * W)", "return fac.V @ (fac.S[:, None] * W)",
     "Sigma instead of Sigma^+ in the apply"),
    ("fastpi", "U_orig = U[reo.row_pos]", "U_orig = U[reo.row_order]", "row permutation in the wrong direction"),
    ("fastpi", "V_orig = V[reo.col_pos]", "V_orig = V[reo.col_order]",
     "column permutation in the wrong direction"),
    ("fastpi", "order = np.lexsort((np.arange(s.size), -s))", "order = np.lexsort((np.arange(s.size), s))",
     "truncation keeps the smallest singular values"),
    ("fastpi", "        keep = _truncate(sig1, s)\n", "        keep = np.arange(s)\n",
     "row phase starts from the first s block triplets, not the largest"),
    ("reorder", "hubs_T = ids_T[np.lexsort((ids_T, -degT[ids_T]))][:m_hub]",
     "hubs_T = ids_T[np.lexsort((-ids_T, -degT[ids_T]))][:m_hub]", "hub ties to the higher id"),
    ("reorder", "hubs_F = ids_F[np.lexsort((ids_F, -degF[ids_F]))][:n_hub]",
     "hubs_F = ids_F[np.lexsort((ids_F, degF[ids_F]))][:n_hub]", "feature hubs of lowest degree"),
    ("reorder", "return int(math.ceil(k * float(n_inst))), int(math.ceil(k * float(n_feat)))",
     "return max(1, int(math.floor(k * float(n_inst)))), int(math.ceil(k * float(n_feat)))",
     "instance hub count rounded down"),
    ("reorder", "        e_act = act_T[rows] & act_F[cols]\n", "        e_act = np.ones(rows.size, dtype=bool)\n",
     "degrees in the original graph, not the current one"),
    ("reorder", "best = np.lexsort((labs, -counts))[0]", "best = np.lexsort((-labs, -counts))[0]",
     "giant component ties to the larger label"),
    ("reorder", "sel_T = sel_T[np.lexsort((sel_T, lab_T[sel_T]))]",
     "sel_T = sel_T[np.lexsort((-sel_T, lab_T[sel_T]))]", "instances of a spoke block in descending id"),
    ("reorder", "        if gI < m_hub or gF < n_hub:\n", "        if gI < m_hub and gF < n_hub:\n",
     "stop only when both sides are short of hubs"),
    ("reorder", "        for h in hubs_T:\n", "        for h in hubs_T[::-1]:\n",
     "first instance hub gets the lowest hub id"),
    ("pinv", "inv = np.where(s > tau, 1.0 / np.where(s > tau, s, 1.0), 0.0)",
     "inv = np.where(s > tau, s, 0.0)", "dense pseudoinverse: Sigma instead of Sigma^+"),
    ("pinv", "        U, s, Vt = U[:, :r], s[:r], Vt[:r]\n", "        pass\n",
     "dense rank-r solve not truncated"),
]


def _plant(index: int) -> None:
    """Install oracle.<module> with mistake `index` planted (runner side)."""
    import types

    sys.path.insert(0, ROOT)
    import oracle

    name, old, new, _ = MUTANTS[index]
    path = os.path.join(ROOT, "oracle", name + ".py")
    with open(path) as fh:
        src = fh.read()
    if src.count(old) != 1:
        raise SystemExit(f"mutant {index}: original text found {src.count(old)} times")
    mod = types.ModuleType("oracle." + name)
    mod.__file__ = path
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    setattr(oracle, name, mod)


# the pin problems are small: one BLAS thread per subprocess, several at once
_ENV = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def _run(index: int) -> subprocess.CompletedProcess:
    return subprocess.run([sys.executable, os.path.abspath(__file__), str(index)], cwd=ROOT, env=_ENV,
                          capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes():
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(zip(range(len(MUTANTS)), ex.map(_run, range(len(MUTANTS)))))


def test_unmutated_pins_pass():
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                       env=_ENV, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("index", range(len(MUTANTS)), ids=[m[3] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, index):
    r = outcomes[index]
    # exit code 1: the pin files ran and at least one test failed (not a
    # collection or usage error, which would be 2 or more)
    assert r.returncode == 1, f"mistake not caught (exit {r.returncode}):\n{r.stdout[-1500:]}{r.stderr[-1500:]}"


if __name__ == "__main__":
    _plant(int(sys.argv[1]))
    import pytest as _pt
    sys.exit(_pt.main(["-q", "-x", "-p", "no:cacheprovider", *PINS]))
