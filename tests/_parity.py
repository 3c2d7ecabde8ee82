"""Per-particle accuracy bars shared by the GPU parity tests.

Against the FP64 oracle on identical lists:
- plain FP64 form: acceleration, jerk and potential within 1e-11 relative for
  every particle (reordered FP64 sums of up to ~1e4 terms);
- mixed form: acceleration and potential <= 1e-6 relative for every particle;
  jerk <= 1e-5 relative for every particle, except that a particle whose jerk
  nearly cancels may instead satisfy |error| <= 1e-6 J_scale, where
  J_scale = sum_j m_j (|w| s^-3/2 + 3 |r.w| |r| s^-5/2) is the size of the
  terms its jerk sums.  No quantile: every particle is bounded.
"""
import numpy as np

FP64_REL = 1e-11
MIX_ACC = 1e-6
MIX_POT = 1e-6
MIX_JERK = 1e-5
MIX_JERK_SCALED = 1e-6


def errors(acc, jerk, pot, ra, rj, rp):
    """Relative errors per particle; acc, jerk are [3, k] (GPU), ra, rj [k, 3] (oracle)."""
    ea = np.linalg.norm(acc.T - ra, axis=1) / np.linalg.norm(ra, axis=1)
    ej = np.linalg.norm(jerk.T - rj, axis=1) / np.linalg.norm(rj, axis=1)
    ep = np.abs(pot - rp) / np.abs(rp)
    return ea, ej, ep


def jscale(xj, vj, mj, gid, off, idx, i_idx, eps2):
    """J_scale of each particle i_idx[k] over its list (group gid[k]), self skipped."""
    out = np.zeros(len(i_idx))
    for k, i in enumerate(i_idx):
        g = gid[k]
        lst = idx[off[g]:off[g + 1]]
        lst = lst[lst != i]
        r = xj[lst] - xj[i]
        w = vj[lst] - vj[i]
        s = (r * r).sum(1) + eps2
        rw = np.abs((r * w).sum(1))
        out[k] = (mj[lst] * (np.linalg.norm(w, axis=1) * s ** -1.5
                             + 3 * rw * np.linalg.norm(r, axis=1) * s ** -2.5)).sum()
    return out


def check(fp64, acc, jerk, pot, ra, rj, rp, jscale_of=None, label=""):
    """Asserts the bars for every particle and prints the maxima.  jscale_of(k)
    returns J_scale for the particles at positions k (needed for the mixed form
    when some jerk error exceeds 1e-5)."""
    ea, ej, ep = errors(acc, jerk, pot, ra, rj, rp)
    print(f"\n{label}: acc max {ea.max():.2e}, jerk max {ej.max():.2e}, pot max {ep.max():.2e} "
          f"({len(ea)} particles)")
    if fp64:
        assert ea.max() < FP64_REL, ea.max()
        assert ej.max() < FP64_REL, ej.max()
        assert ep.max() < FP64_REL, ep.max()
        return ea, ej, ep
    assert ea.max() <= MIX_ACC, ea.max()
    assert ep.max() <= MIX_POT, ep.max()
    bad = np.nonzero(ej > MIX_JERK)[0]
    if len(bad):
        assert jscale_of is not None, f"{len(bad)} jerks above {MIX_JERK} and no J_scale to judge them"
        js = jscale_of(bad)
        ejs = np.linalg.norm(jerk.T[bad] - rj[bad], axis=1) / js
        print(f"  {len(bad)} near-cancelling jerks; error / J_scale max {ejs.max():.2e}")
        assert ejs.max() <= MIX_JERK_SCALED, ejs.max()
    return ea, ej, ep
