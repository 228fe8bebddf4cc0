"""The oracle's pins catch plausible mistakes.  Each case plants one mistake (a dropped term,
a flipped sign, a wrong operand or index) in a copy of the oracle's C source, compiles it on
the CPU, and runs the pin suites against it in a subprocess: at least one pin must fail.
The GB300 library is not involved."""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mps_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_options.py",
        "tests/test_oracle_two_phase.py", "tests/test_oracle_adjoint.py"]

MUTATIONS = [
    ("weight: the -1 of Eq. 4 dropped", "    return re / r - 1.0;\n}", "    return re / r;\n}"),
    ("squared distance: wrong operand", "    s = s + dz * dz;", "    s = s + dy * dz;"),
    ("neighbour predicate: r <= re", "    return dist2(xj - xi, yj - yi, zj - zi) < re2;",
     "    return dist2(xj - xi, yj - yi, zj - zi) <= re2;"),
    ("lambda: r^4 for r^2", "                swr2 = swr2 + w * r2;",
     "                swr2 = swr2 + w * r2 * r2;"),
    ("Laplacian: d for 2d", "    double coef = (2.0 * dim) / (n0 * lambda);",
     "    double coef = (1.0 * dim) / (n0 * lambda);"),
    ("Laplacian: flipped difference",
     "                    s = s + (phi[j * ncomp + c] - phi[i * ncomp + c]) * w;",
     "                    s = s + (phi[i * ncomp + c] - phi[j * ncomp + c]) * w;"),
    ("gradient: r_i - r_j",
     "                double d[3] = {xj - xi, yj - yi, zj - zi};\n"
     "                double r2 = dist2(d[0], d[1], d[2]);\n"
     "                double w = weight(sqrt(r2), re, kernel);",
     "                double d[3] = {xi - xj, yi - yj, zi - zj};\n"
     "                double r2 = dist2(d[0], d[1], d[2]);\n"
     "                double w = weight(sqrt(r2), re, kernel);"),
    ("PPE: diagonal term dropped", "        A->val[k0] = diag + p->alpha_c / (p->dt * p->dt);",
     "        A->val[k0] = diag;"),
    ("PPE: off-diagonal sign", "                A->val[k] = -c;", "                A->val[k] = c;"),
    ("PPE: right-hand side sign",
     "        b[i] = in_ppe(type, flags, i) ? inv_dt2 * ((nstar[i] - n0) / n0) : 0.0;",
     "        b[i] = in_ppe(type, flags, i) ? inv_dt2 * ((n0 - nstar[i]) / n0) : 0.0;"),
    ("predict: gravity dropped",
     "                    us[q] = vel[q] + p->dt * (nu_of(p, i) * lap[q] + p->g[a]);",
     "                    us[q] = vel[q] + p->dt * (nu_of(p, i) * lap[q]);"),
    ("correction: position update without dt", "                pos[q] = ps[q] + p->dt * du;",
     "                pos[q] = ps[q] + du;"),
    ("free surface: n* <= beta n0 turned around",
     "&& nstar[i] < p->beta * R->n0_pnd;", "&& nstar[i] > p->beta * R->n0_pnd;"),
    ("equation of state: exponent gamma - 1", "(pow(nstar / n0, p->gamma) - 1.0)",
     "(pow(nstar / n0, p->gamma - 1.0) - 1.0)"),
    ("two-phase: the row's density for the pair",
     "(coef0 * (2.0 / (p->rho_i[i] + p->rho_i[j]))) * w", "(coef0 * (1.0 / p->rho_i[i])) * w"),
    ("cubic kernel: square for cube", "        return t * t * t;", "        return t * t;"),
    ("CMPS: p_hat_j replaced by p_hat_i", "((p[i] + p[j]) - (phat[i] + phat[j]))",
     "((p[i] + p[j]) - (phat[i] + phat[i]))"),
    ("HS: sign of Dn/Dt", "        out[i] = -s;", "        out[i] = s;"),
    ("gradient: 1/n0 for d/n0",
     "        for (int a = 0; a < dim; a++) out[i * dim + a] = ((double)dim / n0) * s[a];",
     "        for (int a = 0; a < dim; a++) out[i * dim + a] = (1.0 / n0) * s[a];"),
    ("PPE: surface neighbours left off the diagonal (p_j = 0 not imposed)",
     "            diag = diag + c;\n            if (in_ppe(type, flags, j)) {\n"
     "                A->col[k] = (int32_t)j;",
     "            if (in_ppe(type, flags, j)) {\n                diag = diag + c;\n"
     "                A->col[k] = (int32_t)j;"),
    ("PPE: dummy neighbours taken as coefficients",
     "            if (type[j] == ORC_DUMMY) continue;\n            double xj, yj, zj;\n"
     "            coords(pos, dim, j, &xj, &yj, &zj);\n"
     "            double w = weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), p->re_lap, p->kernel);",
     "            double xj, yj, zj;\n"
     "            coords(pos, dim, j, &xj, &yj, &zj);\n"
     "            double w = weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), p->re_lap, p->kernel);"),
    ("predict: r* from the old velocity", "                    ps[q] = pos[q] + p->dt * us[q];",
     "                    ps[q] = pos[q] + p->dt * vel[q];"),
    ("free surface: walls never on it",
     "        int surf = (type[i] == ORC_FLUID || type[i] == ORC_WALL) && nstar[i] <",
     "        int surf = (type[i] == ORC_FLUID) && nstar[i] <"),
    ("number density: dummies left out",
     "                coords(pos, dim, j, &xj, &yj, &zj);\n"
     "                s = s + weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), re, kernel);",
     "                if (type[j] == ORC_DUMMY) continue;\n"
     "                coords(pos, dim, j, &xj, &yj, &zj);\n"
     "                s = s + weight(sqrt(dist2(xj - xi, yj - yi, zj - zi)), re, kernel);"),
    ("equation of state: surface particles keep their pressure",
     "            pres[i] = in_ppe(type, flags, i) ? wc_pressure(p, rho_of(p, i), nstar[i], n0)"
     " : 0.0;\n            phat[i] = pres[i];",
     "            pres[i] = (type[i] == ORC_FLUID || type[i] == ORC_WALL) ?"
     " wc_pressure(p, rho_of(p, i), nstar[i], n0) : 0.0;\n            phat[i] = pres[i];"),
    ("two-phase: correction with the reference density",
     "                double du = -(p->dt / rho_of(p, i)) * grad[q];",
     "                double du = -(p->dt / p->rho) * grad[q];"),
    ("ghost: velocity kept",
     "                for (int a = 0; a < p->dim; a++) vel[i * p->dim + a] = 0.0;", ""),
    ("Dn/Dt: one power of r dropped", "                s = s + p->re_n / (r2 * r) * dot;",
     "                s = s + p->re_n / r2 * dot;"),
    ("HS: ECS without its first term",
     "            double ecs = fabs(eps) * (dk[i] / n0) + fabs(p->dt * dk[i] / n0) * (eps / p->dt);",
     "            double ecs = fabs(p->dt * dk[i] / n0) * (eps / p->dt);"),
    ("HS: dt missing in b", "        double v = dstar[i] / (n0 * p->dt);",
     "        double v = dstar[i] / n0;"),
    ("clamp ignored on the step",
     "        if (p->clamp_negative_p)\n            for (int64_t i = 0; i < n; i++)\n"
     "                if (pres[i] < 0.0) pres[i] = 0.0;\n"
     "        for (int64_t i = 0; i < n; i++) {\n            double m = pres[i];",
     "        for (int64_t i = 0; i < n; i++) {\n            double m = pres[i];"),
    ("PPE right-hand side: n0 of the Laplacian",
     "            ppe_rhs(p, n, type, flags, nstar, n0, bvec);\n        }\n        rc = cg_solve",
     "            ppe_rhs(p, n, type, flags, nstar, R.n0_lap, bvec);\n        }\n        rc = cg_solve"),
    ("viscosity: n0 of the number density for that of the Laplacian",
     "laplacian_from(dim, n, pos, type, p->re_lap, p->kernel, R->n0_lap, R->lambda, &nb, vel,",
     "laplacian_from(dim, n, pos, type, p->re_lap, p->kernel, R->n0_pnd, R->lambda, &nb, vel,"),
    ("p_hat: dummies taken into the minimum",
     "                if (type[j] != ORC_DUMMY && pres[j] < m) m = pres[j];\n"
     "            }\n            phat[i] = m;\n        }\n    } else {",
     "                if (pres[j] < m) m = pres[j];\n"
     "            }\n            phat[i] = m;\n        }\n    } else {"),
    ("p_hat: the particle's own p_i left out of the minimum",
     "                if (pres[i] < 0.0) pres[i] = 0.0;\n        for (int64_t i = 0; i < n; i++) {\n"
     "            double m = pres[i];",
     "                if (pres[i] < 0.0) pres[i] = 0.0;\n        for (int64_t i = 0; i < n; i++) {\n"
     "            double m = HUGE_VAL;"),
    ("ECS: signed density deviation", "            double ecs = fabs(eps) * (dk[i] / n0)",
     "            double ecs = eps * (dk[i] / n0)"),
    ("adjoint: sign of the PPE coefficient cotangent",
     "                double gc = -lam[i] * (ppre[i] - ppre[j]);",
     "                double gc = lam[i] * (ppre[i] - ppre[j]);"),
    ("adjoint: viscosity's transpose onto the neighbour dropped",
     "                out_u[j * dim + a] = out_u[j * dim + a] + k * w * gsa;", ""),
    ("adjoint: p_hat path dropped",
     "        if (type[i] == ORC_FLUID) gp[amin[i]] = gp[amin[i]] + gphat[i];", ""),
    ("adjoint: sign of the number-density derivative",
     "            double f = gn[i] * (-p->re_n / s2) / sqrt(s2);",
     "            double f = gn[i] * (p->re_n / s2) / sqrt(s2);"),
    ("adjoint: clamp mask ignored",
     "        else if (p->pressure_mode == 0 && p->clamp_negative_p && !(ppre[i] > 0.0)) gp[i] = 0.0;",
     ""),
    ("adjoint: equation-of-state exponent gamma for gamma - 1",
     "pow(nstar[i] / n0, p->gamma - 1.0) / n0;", "pow(nstar[i] / n0, p->gamma) / n0;"),
    ("adjoint: r* = r + dt u* path dropped",
     "                gus[q] = gus[q] + dt * grs[q];", ""),
    ("adjoint: right-hand side scale n0 dt for n0 dt^2",
     "            gn[i] = lam[i] / (n0 * dt * dt);", "            gn[i] = lam[i] / (n0 * dt);"),
    ("adjoint: gradient pair term without its radial part",
     "            for (int a = 0; a < 3; a++) X[a] = f * (q * gi[a] + (qd / s) * dg * d[a]);",
     "            for (int a = 0; a < 3; a++) X[a] = f * (q * gi[a]);"),
    ("adjoint: derivative of w/r^2 with r^4 for r^3",
     "            double qd = wd / s2 - 2.0 * w / (s2 * s);",
     "            double qd = wd / s2 - 2.0 * w / (s2 * s2);"),
    ("adjoint: correction cotangent without dt r",
     "            gG[q] = k * (gu[q] + dt * gr[q]);", "            gG[q] = k * gu[q];"),
    ("adjoint: viscosity position term sign",
     "            double f = k * gdu * (-p->re_lap / s2) / s;",
     "            double f = k * gdu * (p->re_lap / s2) / s;"),
]


def _run_mutant(name, old, new, workdir):
    src = open(SRC).read()
    assert src.count(old) == 1, f"anchor of '{name}' not unique"
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)[:40]
    c_path = os.path.join(workdir, f"{tag}.c")
    so_path = os.path.join(workdir, f"{tag}.so")
    open(c_path, "w").write(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                           "-std=c11", "-o", so_path, c_path, "-lm"])
    env = dict(os.environ, MPS_ORACLE_LIB=so_path, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"] + PINS, cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return name, r.returncode


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as d:
        with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
            results = list(ex.map(lambda m: _run_mutant(*m, d), MUTATIONS))
    survived = [name for name, rc in results if rc == 0]
    assert not survived, f"mistakes no pin catches: {survived}"
