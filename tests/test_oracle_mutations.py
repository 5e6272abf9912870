"""Mutation check of the oracle's pins: each plausible mistake below (a
dropped term, a wrong sign, factor or index, a wrong comparison) is planted
in a copy of the oracle's C source, which is rebuilt on its own, and the
oracle's pin files run against the copy; every mistake must make at least
one pin fail.  An unmutated copy must pass them all (the control).  Nothing
here touches the oracle in the tree or any GPU.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_oracle_coupled.py", "tests/test_oracle_open.py"]

# (what the mistake is, text in the oracle's C source, what it becomes[,
# which occurrence of the text, from 0; the first if not given])
MUTATIONS = [
    # the particle update (Sec. 2.2, App. A)
    ("Boris rotation vector without the half step", "b[d] = 0.5 * h * Bp[d] / gam;", "b[d] = h * Bp[d] / gam;"),
    ("rotation without its 1/(1+b^2) factor", "v1[d] = v0[d] + 2.0 * txb[d] / (1.0 + b2);",
     "v1[d] = v0[d] + 2.0 * txb[d];"),
    ("ideal-MHD field with the wrong sign", "E0[d] = -vxb[d];", "E0[d] = vxb[d];", 0),
    ("predictor's ideal-MHD field with the wrong sign", "E0[d] = -vxb[d];", "E0[d] = vxb[d];", 1),
    ("TSC upper weight mirrored", "w[2] = 0.5 * (0.5 + delta) * (0.5 + delta);",
     "w[2] = 0.5 * (0.5 - delta) * (0.5 - delta);"),
    ("parallel field left in", "Ep[d] -= eb * Bp[d];", "Ep[d] -= 0.0 * eb;"),
    ("second drift with the old velocity", "xp[d] = xp[d] + 0.5 * dt * (vnew[d] / g1);",
     "xp[d] = xp[d] + 0.5 * dt * (vn[d] / g0);"),
    ("first half-kick energy change with a difference for the sum", "s0[d] = v0[d] + vn[d];",
     "s0[d] = v0[d] - vn[d];"),
    ("second half-kick energy change without the rotated velocity", "s1[d] = vnew[d] + v1[d];",
     "s1[d] = vnew[d] + v0[d];"),
    ("corrector y-momentum with the wrong sign", "double q[4] = {-m * dv[0], -m * dv[1]",
     "double q[4] = {-m * dv[0], m * dv[1]"),
    ("current from the four-velocity", "q[1 + d] = p->qm_cr * m * (vnew[d] / g1) / dV;",
     "q[1 + d] = p->qm_cr * m * vnew[d] / dV;"),
    ("open box's lower wall folds into the wrong cell", "i = -1 - i;", "i = -i;", 0),
    ("reflecting wall folds into the wrong cell", "i = -1 - i;", "i = -i;", 1),
    ("reflecting upper wall folds into the wrong cell", "i = 2 * n - 1 - i;", "i = 2 * n - 2 - i;"),
    ("gamma with half the momentum term", "return sqrt(C * C + dot3(v, v)) / C;",
     "return sqrt(C * C + 0.5 * dot3(v, v)) / C;"),
    ("kinetic energy over gamma", "return dot3(v, v) / (orc_gamma(v, C) + 1.0);",
     "return dot3(v, v) / orc_gamma(v, C);"),
    ("TSC centre weight", "w[1] = 0.75 - delta * delta;", "w[1] = 0.75 - 0.5 * delta * delta;"),
    ("TSC offset from the cell face, not the centre", "double delta = s - fi - 0.5;", "double delta = s - fi;"),
    ("position in cells without the cell size", "double s = (xp[d] - g->x0[d]) / g->dx[d];",
     "double s = xp[d] - g->x0[d];"),
    ("stencil weight without its y factor", "wts[m] = w[0][a] * w[1][b] * wz;", "wts[m] = w[0][a] * wz;"),
    ("gather without the weights", "acc += wts[k] * planes[q * nc + cells[k]];",
     "acc += planes[q * nc + cells[k]] / m;"),
    ("first drift a full step", "xp[d] = xp[d] + 0.5 * dt * (vn[d] / g0);", "xp[d] = xp[d] + dt * (vn[d] / g0);"),
    ("parallel field kept where |B| = 1", "if (B2 > 0.0) {", "if (B2 > 1.0) {"),
    ("first kick a full step", "v0[d] = vn[d] + 0.5 * h * Ep[d];", "v0[d] = vn[d] + h * Ep[d];"),
    ("second kick a full step", "vnew[d] = v1[d] + 0.5 * h * Ep[d];", "vnew[d] = v1[d] + h * Ep[d];"),
    ("rotation's gamma from the old velocity", "double gam = orc_gamma(v0, C);", "double gam = orc_gamma(vn, C);"),
    ("rotation's inner cross product reversed", "cross3(v0, b, t);", "cross3(b, v0, t);"),
    ("push without the charge-to-mass ratio", "const double h = p->qm_cr * dt;", "const double h = dt;"),
    ("moments' charge without the charge-to-mass ratio", "q[0] = p->qm_cr * p->m_cr / dV;", "q[0] = p->m_cr / dV;"),
    ("push's charge deposit without the charge-to-mass ratio", "q[0] = p->qm_cr * m / dV;", "q[0] = m / dV;"),
    ("upper wall reflection keeps the normal velocity", "xp[d] = 2.0 * hi - xp[d];\n                v[d] = -v[d];",
     "xp[d] = 2.0 * hi - xp[d];\n                v[d] = v[d];"),
    ("leaving particle put outside the open face", "xp[d] = nextafter(hi, lo);\n            left = 1;",
     "xp[d] = hi;\n            left = 1;"),
    ("wall reflection keeps the normal velocity", "xp[d] = 2.0 * lo - xp[d];\n                v[d] = -v[d];",
     "xp[d] = 2.0 * lo - xp[d];\n                v[d] = v[d];"),
    ("periodic wrap by half the box", "r -= L * floor(r / L);", "r -= 0.5 * L * floor(r / L);"),
    # the CR-Hall term and the feedback (Sec. 2.1)
    ("Hall field added", "E[d * nc + c] = E0[d] - F / ng;", "E[d * nc + c] = E0[d] + F / ng;"),
    ("gas charge density without its charge-to-mass ratio", "double ng = p->qm_gas * rho[c];", "double ng = rho[c];", 0),
    ("gas velocity from the momentum density", "vg[d] = mom[d * nc + c] / rho[c];", "vg[d] = mom[d * nc + c];"),
    ("momentum feedback not per cell volume", "mom[d * nc + c] += corr[d * nc + c] / dV;",
     "mom[d * nc + c] += corr[d * nc + c];"),
    ("gas momentum total without the cell volume", "out[d] += mom[d * nc + c] * dV;", "out[d] += mom[d * nc + c];"),
    ("CR energy total from |v|^2/2", "out[7] += p->m_cr * orc_kinetic_energy(vj, p->C);",
     "out[7] += p->m_cr * 0.5 * dot3(vj, vj);"),
    # diagnostics (Sec. 2.2, 4.3)
    ("spectrum puts a value on an edge in the lower bin", "while (b + 1 < nbins && edges[b + 1] <= q)",
     "while (b + 1 < nbins && edges[b + 1] < q)"),
    ("spectrum's upper moment without its last factor", "sums[0] += qn * q;", "sums[0] += qn;"),
    ("spectrum energy over gamma", "q = v2 / (gam + 1.0);", "q = v2 / gam;"),
    ("spectrum region open at its lower edge", "if (!(xd >= region[2 * d] && xd < region[2 * d + 1]))",
     "if (!(xd > region[2 * d] && xd < region[2 * d + 1]))"),
    ("Lambda without the CR density", "lam[d * nc + c] = vA > 0.0 ? (J - n * vg) / ((ng + n) * vA) : 0.0;",
     "lam[d * nc + c] = vA > 0.0 ? (J - n * vg) / (ng * vA) : 0.0;"),
    ("Lambda's gas density without its charge-to-mass ratio", "double ng = p->qm_gas * rho[c];",
     "double ng = rho[c];", 1),
    ("Alfven speed over rho", "double vA = sqrt(dot3(Bc, Bc)) / sqrt(rho[c]);",
     "double vA = sqrt(dot3(Bc, Bc)) / rho[c];"),
    # the CR-Hall term and the feedback (Sec. 2.1), continued
    ("CR fraction without the CR density", "double R = n / (ng + n);", "double R = n / ng;"),
    ("Hall force with J x B of the wrong sign", "double F = (1.0 - R) * (n * E0[d] + JxB[d]);",
     "double F = (1.0 - R) * (n * E0[d] - JxB[d]);"),
    ("energy feedback not per cell volume", "egas[c] += corr[3 * nc + c] / dV;", "egas[c] += corr[3 * nc + c];", 0),
    ("coupled energy feedback not per cell volume", "egas[c] += corr[3 * nc + c] / dV;",
     "egas[c] += corr[3 * nc + c];", 1),
    # the cell sort
    ("scatter in reverse order (not stable)",
     "for (int64_t j = 0; j < np; ++j) {\n        int64_t k = cell[j] < 0",
     "for (int64_t j = np - 1; j >= 0; --j) {\n        int64_t k = cell[j] < 0"),
    ("cells within a brick ordered y before x",
     "int64_t in = ((k % brick[2]) * brick[1] + j % brick[1]) * brick[0] + i % brick[0];",
     "int64_t in = ((k % brick[2]) * brick[0] + i % brick[0]) * brick[1] + j % brick[1];"),
    ("bricks ordered y before x", "int64_t bid = ((k / brick[2]) * nby + j / brick[1]) * nbx + i / brick[0];",
     "int64_t bid = ((k / brick[2]) * nbx + i / brick[0]) * nby + j / brick[1];"),
    ("open face drops the weight beyond it into the wrong cell", "return i >= n ? n - 1 : i;",
     "return i >= n ? n - 2 : i;"),
    # the coupled predictor-corrector step (Sec. 3, App. B.2)
    ("Hall induction with the wrong sign", "dB[nc + c] -= (H[2 * nc + r]", "dB[nc + c] += (H[2 * nc + r]"),
    ("predictor a full step",
     "mom_h[d * nc + c] = mom[d * nc + c] + 0.5 * dt * (dmom[d * nc + c] - F[d * nc + c]);",
     "mom_h[d * nc + c] = mom[d * nc + c] + dt * (dmom[d * nc + c] - F[d * nc + c]);"),
    ("predictor Hall force without (1 - R)", "F[d] = (1.0 - R) * (n * E0[d] + JxB[d]);\n    *P",
     "F[d] = (n * E0[d] + JxB[d]);\n    *P"),
    ("centred difference without the 1/2", "double h = 1.0 / (2.0 * g->dx[0]);", "double h = 1.0 / (g->dx[0]);"),
    ("corrector momentum with the wrong sign", "mom[d * nc + c] += dt * dmom[d * nc + c] + corr[d * nc + c] / dV;",
     "mom[d * nc + c] += dt * dmom[d * nc + c] - corr[d * nc + c] / dV;"),
    ("induction a half step", "B[d * nc + c] += dt * dB[d * nc + c];", "B[d * nc + c] += 0.5 * dt * dB[d * nc + c];"),
    ("corrector source with the wrong sign", "(-corr[d * nc + c] / (dV * dt))", "(corr[d * nc + c] / (dV * dt))"),
    ("one-sided difference", "dB[d * nc + c] = Bx * (mom[d * nc + r] / rho[r] - mom[d * nc + l] / rho[l]) * h;",
     "dB[d * nc + c] = Bx * (mom[d * nc + r] / rho[r] - mom[d * nc + c] / rho[c]) * h;"),
    ("predictor energy source with the wrong sign", "egas_h[c] = egas[c] - 0.5 * dt * P[c];",
     "egas_h[c] = egas[c] + 0.5 * dt * P[c];"),
    ("gas momentum driven by dB_y for both components", "dmom[d * nc + c] = Bx * (B[d * nc + r] - B[d * nc + l]) * h;",
     "dmom[d * nc + c] = Bx * (B[nc + r] - B[nc + l]) * h;"),
    ("Hall induction's z part with the wrong sign", "dB[2 * nc + c] += (H[nc + r] - H[nc + l]) * h;",
     "dB[2 * nc + c] -= (H[nc + r] - H[nc + l]) * h;"),
    ("predictor's Hall field without the gas charge-to-mass ratio",
     "H[d * nc + c] = p->hall ? Fc[d] / (p->qm_gas * rho[c]) : 0.0;", "H[d * nc + c] = p->hall ? Fc[d] / rho[c] : 0.0;"),
    ("predictor's B a full step", "B_h[d * nc + c] = B[d * nc + c] + 0.5 * dt * dB[d * nc + c];",
     "B_h[d * nc + c] = B[d * nc + c] + dt * dB[d * nc + c];"),
    ("source power without (1 - R)", "*P = (1.0 - R) * dot3(J, E0);", "*P = dot3(J, E0);"),
    ("periodic x neighbour off by one", "int64_t j = (i + s + nx) % nx;", "int64_t j = (i + 2 * s + nx) % nx;"),
    # the open face, front tracking and injection (Sec. 5)
    ("front smoothing kernel's width squared dropped", "double w = exp(-0.5 * (double)(k * k) / (sig * sig));",
     "double w = exp(-0.5 * (double)(k * k) / sig);"),
    ("front smoothing not renormalised", "sv[i] = a / ws;", "sv[i] = a;"),
    ("upstream taken from the first cell", "double vup = sv[nx - 1], rup = sr[nx - 1];",
     "double vup = sv[nx - 1], rup = sr[0];"),
    ("front crossing interpolated from the wrong cell", "double f = (thr - a) / (b - a);",
     "double f = (thr - b) / (a - b);"),
    ("front position a cell centre too far", "xs = g->x0[0] + ((double)i + 0.5 + f) * g->dx[0];",
     "xs = g->x0[0] + ((double)i + 1.5 + f) * g->dx[0];"),
    ("jump pressure without the compression factor", "double P1 = r / (r - 1.0) * rup * vup * vup;",
     "double P1 = rup * vup * vup;"),
    ("tail at the cell's lower face", "xt = g->x0[0] + ((double)i + 0.5) * g->dx[0];",
     "xt = g->x0[0] + ((double)i) * g->dx[0];"),
    ("injection direction cosine from [0, 1)", "double mu = 2.0 * unit_open(u[2]) - 1.0;",
     "double mu = unit_open(u[2]);"),
    ("injection azimuth over half a turn", "double ph = 6.283185307179586 * unit_open(u[3]);",
     "double ph = 3.141592653589793 * unit_open(u[3]);"),
    ("injected speed from gamma, not four-velocity", "double vmag = C * sqrt(gp * gp - 1.0);",
     "double vmag = C * sqrt(1.0 - 1.0 / (gp * gp));"),
    ("injected y positions over half the box", "x_new[cap + k] = g->x0[1] + unit_open(u[0]) * g->n[1] * g->dx[1];",
     "x_new[cap + k] = g->x0[1] + 0.5 * unit_open(u[0]) * g->n[1] * g->dx[1];"),
    ("injected energy removed from the gas twice", "egas[c] -= Ein / Vreg;", "egas[c] -= 2.0 * Ein / Vreg;"),
    ("front speed from one step only", "double V = isnan(xs_prev) ? 0.0 : (xs - xs_prev) / dt;",
     "double V = isnan(xs_prev) ? 0.0 : (xs - xs_prev) / (2.0 * dt);"),
    ("front smoothing width", "const double sig = 4.0;", "const double sig = 3.0;"),
    ("front threshold", "double thr = 0.6 * fabs(vup);", "double thr = 0.4 * fabs(vup);"),
    ("injected mass added to the gas", "rho[c] -= Min / Vreg;", "rho[c] += Min / Vreg;"),
    ("boost of the injected particles backwards", "vv[0] = Gam * (vv[0] + V * gp);", "vv[0] = Gam * (vv[0] - V * gp);"),
    ("generator without the key word", "uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;",
     "uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1;"),
    ("injection energy without the 1/2", "double Ek = energy_factor * 0.5 * vup * vup;",
     "double Ek = energy_factor * vup * vup;"),
    ("fractional particle count dropped", "double want = eta * M / p->m_cr + *carry;", "double want = eta * M / p->m_cr;"),
    ("half the injected momentum taken from the gas", "mom[d * nc + c] -= Pin[d] / Vreg;",
     "mom[d * nc + c] -= 0.5 * Pin[d] / Vreg;"),
    ("shocked region threshold", "if (sp[i] >= (2.0 / 3.0) * P1) {", "if (sp[i] >= (1.0 / 3.0) * P1) {"),
    ("swept mass without the front speed", "double M = rup * (fabs(vup) + (V > 0.0 ? V : 0.0)) * dt * A;",
     "double M = rup * fabs(vup) * dt * A;"),
    ("open face a cell late", "if (g->bc[d] == 2 && xp[d] >= hi) {", "if (g->bc[d] == 2 && xp[d] > hi + 1.0) {"),
    # early-particle removal (Sec. 5)
    ("removal includes the threshold time", "if (t_inj[j] < t_early && t >= 2.0 * t_inj[j]) {",
     "if (t_inj[j] <= t_early && t >= 2.0 * t_inj[j]) {"),
    ("removal a step late at exactly twice", "if (t_inj[j] < t_early && t >= 2.0 * t_inj[j]) {",
     "if (t_inj[j] < t_early && t > 2.0 * t_inj[j]) {"),
    ("removal at the injection time, not twice it", "if (t_inj[j] < t_early && t >= 2.0 * t_inj[j]) {",
     "if (t_inj[j] < t_early && t >= t_inj[j]) {"),
]

# the same for the oracle's Python layer (oracle/__init__.py)
PY_MUTATIONS = [
    ("coupled step pushes in the old magnetic field",
     "push(self.g, self.p, dt, self.x, self.v, E, half[3], self.corr, self.mom_dep)",
     "push(self.g, self.p, dt, self.x, self.v, E, self.B, self.corr, self.mom_dep)"),
    ("coupled step keeps the old moments", "        self.mom_dep[:] = 0.0\n        push(", "        push("),
    ("box parameters with the two charge-to-mass ratios swapped",
     "make_params(box.qm_cr, box.qm_gas, box.C, box.m_cr, box.hall)",
     "make_params(box.qm_gas, box.qm_cr, box.C, box.m_cr, box.hall)"),
]


def _mutate(src, name, old, new, nth=0):
    k = -1
    for _ in range(nth + 1):
        k = src.find(old, k + 1)
        assert k >= 0, "not in the oracle: " + name
    return src[:k] + new + src[k + len(old):]


def _run_pins(work, src, py_src):
    """Build the oracle from src in a directory of its own and run the pin
    files against it; pytest's exit code (0 all passed, 1 some failed)."""
    d = os.path.join(work, "oracle")
    os.makedirs(d)
    with open(os.path.join(d, "__init__.py"), "w") as f:
        f.write(py_src)
    with open(os.path.join(d, "mhdpic_oracle.c"), "w") as f:
        f.write(src)
    env = dict(os.environ, PYTHONPATH=work + os.pathsep + ROOT, PYTHONDONTWRITEBYTECODE="1")
    subprocess.run([sys.executable, "-c", "import oracle; oracle.build(force=True)"], cwd=work, env=env,
                   check=True, capture_output=True, timeout=300)
    code = ("import os, sys, oracle\n"
            "assert os.path.dirname(oracle.__file__) == %r, oracle.__file__\n"
            "import pytest\n"
            "sys.exit(pytest.main(['-q', '-x', '-p', 'no:cacheprovider', '-m', 'not gpu'] + %r))\n"
            % (d, [os.path.join(ROOT, f) for f in PIN_FILES]))
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=work, env=env, capture_output=True, text=True,
                           timeout=180)
    except subprocess.TimeoutExpired:
        return None, "no result within 180 s"
    return r.returncode, r.stdout[-400:] + r.stderr[-400:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(os.path.join(ROOT, "oracle", "mhdpic_oracle.c")) as f:
        src = f.read()
    with open(os.path.join(ROOT, "oracle", "__init__.py")) as f:
        py_src = f.read()
    jobs = [("control", src, py_src)]
    jobs += [(m[0], _mutate(src, *m), py_src) for m in MUTATIONS]
    jobs += [(m[0], src, _mutate(py_src, *m)) for m in PY_MUTATIONS]
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda k: _run_pins(str(tmp_path / ("m%03d" % k)), jobs[k][1], jobs[k][2]),
                          range(len(jobs))))
    rc0, out0 = res[0]
    assert rc0 == 0, "the unmutated copy fails its pins:\n" + out0
    survived = [(jobs[k][0], res[k][1]) for k in range(1, len(jobs)) if res[k][0] != 1]
    assert not survived, "mistakes no pin catches (or that broke the run): %s" % survived
