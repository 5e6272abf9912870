"""Mutation check of the input recipes' pins: each plausible mistake below is
planted in a copy of the input generators, and the recipe pins must catch
every one (the same runner as the oracle's mutation check).  The generators
hold no arithmetic of the method; what they fix are the workloads' shapes,
counts and distributions.
"""
import os

from tests._mutation import ROOT, check_all, mutate

PIN_FILES = ["tests/test_workloads.py"]

# (what the mistake is, text in workloads.py, what it becomes[, occurrence])
MUTATIONS = [
    ("drift boost backwards", "q[0] = G * (p[0] + V * gam)", "q[0] = G * (p[0] - V * gam)"),
    ("drift boost without its Lorentz factor", "G = 1.0 / math.sqrt(1.0 - V * V / (C * C))", "G = 1.0"),
    ("power law drawn uniform in p", "mag = 1.0 / (1.0 / lo - u * (1.0 / lo - 1.0 / hi))",
     "mag = lo + u * (hi - lo)"),
    ("power law's upper end dropped", "mag = 1.0 / (1.0 / lo - u * (1.0 / lo - 1.0 / hi))",
     "mag = 1.0 / (1.0 / lo - u * (1.0 / lo))"),
    ("mode amplitude not scaled for the random phases", "amp = dB_rms / math.sqrt(nmodes / 2.0)",
     "amp = dB_rms / math.sqrt(nmodes)"),
    ("3-D polarisation not perpendicular to k", "e = np.cross(k, np.array([1.0, 0.0, 0.0]))",
     "e = np.cross(np.array([1.0, 1.0, 1.0]), np.array([1.0, 0.0, 0.0]))"),
    ("2-D wave numbers up to 6", "grid = np.array([(a, b, 0) for a in range(-4, 5) for b in range(-4, 5)",
     "grid = np.array([(a, b, 0) for a in range(-6, 7) for b in range(-6, 7)"),
    ("directions uniform in a cube, not on the sphere", "g = rng.standard_normal((3, m))",
     "g = rng.random((3, m)) - 0.5"),
    ("positions not uniform", "s[d] = n[d] * rng.random(m)", "s[d] = n[d] * rng.random(m) ** 1.05"),
    ("dense layer with 75% of the particles", "n_dense = int(round(dense_frac_parts * total))",
     "n_dense = int(round(0.75 * total))"),
    ("shock inflow away from the wall", "gas = _gas(nn, 1.0, (-20.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0)",
     "gas = _gas(nn, 1.0, (20.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0)"),
    ("downstream pressure 3/4 rho v^2", "P = np.where(down, 4.0 / 3.0 * v0 * v0, 1.0)",
     "P = np.where(down, 0.75 * v0 * v0, 1.0)"),
    ("free slots counted per cell", "nfree = int(round(free_frac * total))", "nfree = int(round(free_frac * nc))"),
    ("Alfvenic gas velocity along dB", "gas = _gas(nn, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, -dB)",
     "gas = _gas(nn, 1.0, (0.0, 0.0, 0.0), B, 1.0, 5.0 / 3.0, dB)", 0),
    ("beam drift at 1 v_A", "kind=\"mono\", C=C, pmag=100.0, V=10.0", "kind=\"mono\", C=C, pmag=100.0, V=1.0"),
    ("ensemble boxes seeded apart from seed0", "rng = _rng(seed0 + b)", "rng = _rng(seed0 * 1000 + b)"),
]


def test_every_planted_recipe_mistake_fails_a_pin(tmp_path):
    pkg = "paper_1412_1087_gb300"
    base = {}
    for name in ("__init__.py", "workloads.py"):
        with open(os.path.join(ROOT, pkg, name)) as f:
            base[name] = f.read()
    jobs = [(m[0], {"workloads.py": mutate(base["workloads.py"], *m)}) for m in MUTATIONS]
    check_all(tmp_path, pkg, base, jobs, PIN_FILES)
