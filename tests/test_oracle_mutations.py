"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the oracle's C++ source -- a dropped
term, a wrong sign, index or comparison, a swapped operand -- builds that copy
in a scratch directory and runs the oracle's pin tests against it; at least
one pin must fail.  The mistakes are planted in the oracle only, on the CPU;
the product library is not involved.  Each case names the step of the method
it breaks (centroid, connectivity, pseudo-angle window, straight-line and
Kalman fits, chi2/ndf and the 3-hit rule, extension, seeding and its
conflicts, termination, learned-rejection features and bfloat16 rounding,
forward tracking, Monte-Carlo truth matching).
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ("test_oracle_mc.py", "test_oracle_cluster.py", "test_oracle_fit.py", "test_oracle_track.py", "test_oracle_mlp.py",
             "test_oracle_forward.py", "test_oracle_bruteforce.py")

# (name, exact source text, replacement[, file]): each text occurs once in its
# file of oracle/ (velo_oracle.cpp unless named)
MUTATIONS = [
    ("centroid without the half-pixel offset",
     "snx[id] += q * (int64_t)(2 * w_col(w) + 1);", "snx[id] += q * (int64_t)(2 * w_col(w));"),
    ("4-connectivity instead of 8",
     "int rr = r + dr, cc = c + dc;", "if (dr != 0 && dc != 0) continue;\n        int rr = r + dr, cc = c + dc;"),
    ("pseudo-angle: wrong sign in the second quadrant",
     "k = 1.0f + (-x) / (y - x);", "k = 1.0f + x / (y - x);"),
    ("window distance without the wrap at 4",
     "if (d > 2.0f) d = 4.0f - d;", "if (d > 4.0f) d = 4.0f - d;"),
    ("straight-line fit: Szz sums dz instead of dz^2",
     "    Sz = Sz + dz;\n    Szz = Szz + dz * dz;", "    Sz = Sz + dz;\n    Szz = Szz + dz;"),
    ("straight-line fit: intercept with the wrong sign",
     "R x = (Sx - tx * Sz) / S0;", "R x = (Sx + tx * Sz) / S0;"),
    ("Kalman start without the process noise",
     "R C11 = (s2 + s2) / (dz0 * dz0) + q;", "R C11 = (s2 + s2) / (dz0 * dz0);"),
    ("Kalman prediction with the wrong sign",
     "X = X + T * dz;", "X = X - T * dz;"),
    ("state ndf = 2n - 3",
     "st[18] = (R)(2 * n - 4);", "st[18] = (R)(2 * n - 3);"),
    ("cut ndf = 2n - 3",
     "float ndf = (float)(2 * n - 4);", "float ndf = (float)(2 * n - 3);"),
    ("3-hit rule inverted",
     "if (n == 3 && !(r <= p->chi2ndf_max_3hit)) continue;", "if (n == 3 && (r <= p->chi2ndf_max_3hit)) continue;"),
    ("extension extrapolates from the older hit",
     "float xp = H.x[a] + tx * (Z[m] - H.z[a]);", "float xp = H.x[b] + tx * (Z[m] - H.z[a]);"),
    ("extension takes used hits",
     "        if (used0[h]) continue;\n", ""),
    ("extension contention: largest key wins",
     "claim[bh] = std::min(claim[bh], k);", "claim[bh] = claim[bh] == ~0ull ? k : std::max(claim[bh], k);"),
    ("termination one module late",
     "if (l - m - 1 > (int)p->max_skipped)", "if (l - m - 2 > (int)p->max_skipped)"),
    ("seeding lever arm from the wrong module",
     "float dz12 = H.z[h1] - H.z[h2];", "float dz12 = H.z[h0] - H.z[h1];"),
    ("seeding slope with the wrong denominator",
     "float tx = (H.x[h0] - H.x[h2]) / dz02;", "float tx = (H.x[h0] - H.x[h2]) / (H.z[h0] - H.z[h1]);"),
    ("seeding tie goes to the larger h0",
     "(s == best.s && (h0 < best.h0 ||", "(s == best.s && (h0 > best.h0 ||"),
    ("seeding uses used h0",
     "        if (used[h0]) continue;\n", ""),
    ("seeding h2 window measured from h0",
     "if (dmod4(H.key[h2], H.key[h1]) > p->win_seed) continue;",
     "if (dmod4(H.key[h2], H.key[h0]) > p->win_seed) continue;"),
    ("seeding scatter against the extension cut",
     "if (s > p->max_scatter_seed) continue;", "if (s > p->max_scatter_fwd) continue;"),
    ("extension window centred on the older hit",
     "if (dmod4(H.key[h], H.key[a]) > p->win_fwd) continue;", "if (dmod4(H.key[h], H.key[b]) > p->win_fwd) continue;"),
    ("seed survives without its h2 claim",
     "if (sclaim[s.h0] != k || sclaim[s.h2] != k) continue;", "if (sclaim[s.h0] != k) continue;"),
    ("bfloat16 rounding half away from zero",
     "u += 0x7FFFu + ((u >> 16) & 1u);", "u += 0x8000u;"),
    ("feature RMS without the square root",
     "f[8] = std::sqrt(sxx / fn);", "f[8] = sxx / fn;"),
    ("forward: q/p with the wrong sign",
     "so[0] = have ? (b_b - tx) / geo->kappa : 0.0f;", "so[0] = have ? (tx - b_b) / geo->kappa : 0.0f;"),
    ("forward: chi2 over n - 1",
     "const float rchi = chi2 / (float)(n - 2);", "const float rchi = chi2 / (float)(n - 1);"),
    ("forward: match distance without y",
     "const float ad = d * d + dy * dy;", "const float ad = d * d;"),
    ("forward: far stations from the kick line",
     "hl[L] = nearest(L, a1 + b1 * (geo->z_layers[L] - geo->z_layers[0]), ym + ty * dzl, p->tol_x_far);",
     "hl[L] = nearest(L, xm + tk * dzl, ym + ty * dzl, p->tol_x_far);"),
    ("forward: fewer hits preferred",
     "const bool better = !have || n > b_n ||", "const bool better = !have || n < b_n ||"),
    ("forward: nearest-hit tie to the larger id",
     "if (!f || d < bd || (d == bd && h < bh)) { f = true; bd = d; bh = (uint32_t)h; }\n          }\n          return bh;",
     "if (!f || d < bd || (d == bd && h > bh)) { f = true; bd = d; bh = (uint32_t)h; }\n          }\n          return bh;"),
    ("forward: a NaN distance passes the hit window",
     "if (!(d <= tol) || !(std::fabs(y[h] - yp) <= p->tol_y)) continue;",
     "if (d > tol || std::fabs(y[h] - yp) > p->tol_y) continue;"),
    ("forward: line from the two most upstream hits",
     "const uint32_t ha = track_hits[track_hit_offsets[t + 1] - 1], hb = track_hits[track_hit_offsets[t + 1] - 2];",
     "const uint32_t ha = track_hits[track_hit_offsets[t] + 1], hb = track_hits[track_hit_offsets[t]];"),
    # Monte-Carlo truth matching (efficiency, ghost and clone rates)
    ("truth: a track matches above 70 % instead of at 70 %",
     "if cnt[j] >= min_frac * len(hits):", "if cnt[j] > min_frac * len(hits):", "mc.py"),
    ("truth: 70 % of the truth-carrying hits instead of all hits",
     "if cnt[j] >= min_frac * len(hits):", "if cnt[j] >= min_frac * int((t >= 0).sum()):", "mc.py"),
    ("truth: reconstructible with 2 modules",
     "recon[p] = len(mods) >= 3", "recon[p] = len(mods) >= 2", "mc.py"),
    ("truth: reconstructible by clusters instead of distinct modules",
     "mods = np.unique(cluster_module[ct == p])", "mods = cluster_module[ct == p]", "mc.py"),
    ("truth: charge ties go to the larger id",
     "if s > bestq[c]:", "if s >= bestq[c]:", "mc.py"),
    ("truth: a particle beats noise in a charge tie",
     "if s > bestq[c]:", "if s > bestq[c] or (s == bestq[c] and best[c] < 0 <= p):", "mc.py"),
    ("truth: cluster truth by pixel count instead of summed charge",
     "q = ((words >> 27) & 15).astype(np.int64)", "q = np.ones(len(words), np.int64)", "mc.py"),
    ("truth: clone rate over tracks",
     "clone_rate=n_clone / max(n_matched_p, 1),", "clone_rate=n_clone / max(n_tracks, 1),", "mc.py"),
    ("truth: efficiency counts matched particles that are not reconstructible",
     "n_eff += int(rec[uniq].sum()) if len(uniq) else 0", "n_eff += len(uniq)", "mc.py"),
]


def _run_case(case, scratch):
    name, old, new = case[:3]
    fname = case[3] if len(case) > 3 else "velo_oracle.cpp"
    work = os.path.join(scratch, "case%02d" % MUTATIONS.index(case))
    os.makedirs(os.path.join(work, "tests"))
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(work, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__", "liboracle.so*"))
    shutil.copytree(os.path.join(ROOT, "velogen"), os.path.join(work, "velogen"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    for f in ("conftest.py", "_compare.py") + PIN_TESTS:
        shutil.copy2(os.path.join(ROOT, "tests", f), os.path.join(work, "tests", f))
    shutil.copy2(os.path.join(ROOT, "pytest.ini"), os.path.join(work, "pytest.ini"))
    src = os.path.join(work, "oracle", fname)
    text = open(src).read()
    assert text.count(old) == 1, f"{name}: the source text is not unique"
    open(src, "w").write(text.replace(old, new))
    env = dict(os.environ, PYTHONPATH=work, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"]
                       + [os.path.join("tests", f) for f in PIN_TESTS], cwd=work, env=env,
                       capture_output=True, text=True, timeout=600)
    failed = [ln.split(" ")[1] for ln in r.stdout.splitlines() if ln.startswith("FAILED ")]
    return name, r.returncode, failed, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as scratch:
        with concurrent.futures.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
            results = list(ex.map(lambda c: _run_case(c, scratch), MUTATIONS))
    survivors = [(name, out) for name, rc, failed, out in results if rc == 0]
    for name, rc, failed, out in results:
        print(f"{name}: {'caught by ' + ', '.join(failed) if rc != 0 else 'NOT CAUGHT'}")
    assert not survivors, "mistakes no pin catches: " + "; ".join(n for n, _ in survivors)
