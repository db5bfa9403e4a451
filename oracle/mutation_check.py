"""Mutation check of the C oracle's pins (test infrastructure, not part of the
library).

Each entry plants one plausible mistake in ``fr_oracle.c`` (a wrong constant,
sign, index, weight or dropped term) in a scratch copy of ``oracle/`` and
``tests/`` and runs the pin tests (``tests/test_oracle_pins.py``) against it;
a mistake that no pin catches is reported as a survivor.  The one expected
survivor is ``coarse rho = 1``: the coarse-level density terms cancel between
L^H(u^H) and L^H(R u^h) in the FAS right-hand side (Sec. V.B.2), so that
mutant computes the same result and no test can tell it apart.

    python oracle/mutation_check.py --workdir <scratch folder> [name ...]
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, original text of fr_oracle.c, mistaken text)
MUTANTS = [
 ("ct", "m->ct = 299792.458 / (100.0 * box);", "m->ct = 299792.458 / (10.0 * box);"),
 ("k1", "double k1 = 3.0 * (1.0 + 4.0 * m->ol / om);", "double k1 = 3.0 * (1.0 + 3.0 * m->ol / om);"),
 ("xi pow", "m->xi = fr0 * pow(k1, nhs + 1.0) / nhs;", "m->xi = fr0 * pow(k1, nhs) / nhs;"),
 ("ka a^-3", "double ka = 3.0 * (pow(a, -3.0) + 4.0 * m->ol / om);", "double ka = 3.0 * (pow(a, -2.0) + 4.0 * m->ol / om);"),
 ("src /3", "pow(nhs * a * a * m->xi, 1.0 / (nhs + 1.0)) / 3.0;", "pow(nhs * a * a * m->xi, 1.0 / (nhs + 1.0)) / 2.0;"),
 ("src a^4", "m->src = om * pow(a, 4.0)", "m->src = om * pow(a, 3.0)"),
 ("bkg a^4", "m->bkg = om * pow(a, 4.0)", "m->bkg = om * pow(a, 3.0)"),
 ("bkg 4OL", "m->bkg = om * pow(a, 4.0) * (pow(a, -3.0) + 4.0 * m->ol / om);", "m->bkg = om * pow(a, 4.0) * (pow(a, -3.0) + 3.0 * m->ol / om);"),
 ("dens", "m->dens = om * a;", "m->dens = om;"),
 ("ubar a^2", "m->ubar = log(nhs * a * a * m->xi / pow(ka, nhs + 1.0));", "m->ubar = log(nhs * a * m->xi / pow(ka, nhs + 1.0));"),
 ("ubar pow", "m->ubar = log(nhs * a * a * m->xi / pow(ka, nhs + 1.0));", "m->ubar = log(nhs * a * a * m->xi / pow(ka, nhs));"),
 ("pre hier", "L->pre = H->m.ct * H->m.ct / (2.0 * hh * hh);", "L->pre = H->m.ct * H->m.ct / (hh * hh);"),
 ("pre wrap", "L->pre = m->ct * m->ct / (2.0 * h * h);", "L->pre = m->ct * m->ct / (h * h);"),
 ("flux sign", "flux += (bi + bj) * (uj - ui);", "flux += (bi + bj) * (ui - uj);"),
 ("flux prod", "flux += (bi + bj) * (uj - ui);", "flux += 2.0 * sqrt(bi * bj) * (uj - ui);"),
 ("flux bi only", "flux += (bi + bj) * (uj - ui);", "flux += (2.0 * bi) * (uj - ui);"),
 ("dflux sign", "dflux += bi * (uj - ui) - (bi + bj);", "dflux += bi * (uj - ui) + (bi + bj);"),
 ("dflux bj", "dflux += bi * (uj - ui) - (bi + bj);", "dflux += bj * (uj - ui) - (bi + bj);"),
 ("dflux drop", "dflux += bi * (uj - ui) - (bi + bj);", "dflux += - (bi + bj);"),
 ("ghost r sign", "double ug = ubv - r * ubv + r * ui;", "double ug = ubv - r * ubv - r * ui;"),
 ("ghost ub", "double ug = ubv - r * ubv + r * ui;", "double ug = ubv + r * ui;"),
 ("ghost flux", "flux += (bi + bg) * (ug - ui);", "flux += (bi + bg) * (ubv - ui);"),
 ("ghost dflux1", "dflux += (bi + r * bg) * (ug - ui) + (bi + bg) * (r - 1.0);", "dflux += (bi + bg) * (ug - ui) + (bi + bg) * (r - 1.0);"),
 ("ghost dflux2", "dflux += (bi + r * bg) * (ug - ui) + (bi + bg) * (r - 1.0);", "dflux += (bi + r * bg) * (ug - ui) + (bi + bg) * (r + 1.0);"),
 ("ghost r=1", "const double r = -1.0;", "const double r = -0.5;"),
 ("s exponent", "double s = exp(-ui / (m->nhs + 1.0));", "double s = exp(-ui / (m->nhs + 2.0));"),
 ("s sign", "double s = exp(-ui / (m->nhs + 1.0));", "double s = exp(ui / (m->nhs + 1.0));"),
 ("L dens sign", "*Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) + m->src * s - m->bkg;", "*Lval = L->pre * flux + m->dens * (L->rho[ci] - 1.0) + m->src * s - m->bkg;"),
 ("L rho-1", "*Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) + m->src * s - m->bkg;", "*Lval = L->pre * flux - m->dens * (L->rho[ci]) + m->src * s - m->bkg;"),
 ("L src sign", "*Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) + m->src * s - m->bkg;", "*Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) - m->src * s - m->bkg;"),
 ("L bkg drop", "*Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) + m->src * s - m->bkg;", "*Lval = L->pre * flux - m->dens * (L->rho[ci] - 1.0) + m->src * s;"),
 ("dL sign", "*dL = L->pre * dflux - m->src * s / (m->nhs + 1.0);", "*dL = L->pre * dflux + m->src * s / (m->nhs + 1.0);"),
 ("dL div", "*dL = L->pre * dflux - m->src * s / (m->nhs + 1.0);", "*dL = L->pre * dflux - m->src * s;"),
 ("resid f sign", "d[ci] = lv - (L->f ? L->f[ci] : 0.0);", "d[ci] = lv + (L->f ? L->f[ci] : 0.0);"),
 ("newton sign", "double du = -(lv - (L->f ? L->f[ci] : 0.0)) / dl;", "double du = (lv - (L->f ? L->f[ci] : 0.0)) / dl;"),
 ("newton f", "double du = -(lv - (L->f ? L->f[ci] : 0.0)) / dl;", "double du = -(lv) / dl;"),
 ("restrict /8", "coarse[idx3(nc, I, J, K)] = s / 8.0;", "coarse[idx3(nc, I, J, K)] = s / 4.0;"),
 ("restrict idx", "s += fine[idx3(nf, 2 * I + a, 2 * J + b, 2 * K + c)];", "s += fine[idx3(nf, 2 * I + a, 2 * J + b, 2 * K)];"),
 ("restrict swap", "s += fine[idx3(nf, 2 * I + a, 2 * J + b, 2 * K + c)];", "s += fine[idx3(nf, 2 * J + a, 2 * I + b, 2 * K + c)];"),
 ("rfaces /4", "ubc[oc[f] + (long)Q * nc[p] + P] = s / 4.0;", "ubc[oc[f] + (long)Q * nc[p] + P] = s / 2.0;"),
 ("rfaces transp", "s += ubf[of[f] + (long)(2 * Q + b) * nf[p] + (2 * P + a)];", "s += ubf[of[f] + (long)(2 * P + b) * nf[p] + (2 * Q + a)];"),
 ("rfaces one", "s += ubf[of[f] + (long)(2 * Q + b) * nf[p] + (2 * P + a)];", "s += ubf[of[f] + (long)(2 * Q) * nf[p] + (2 * P + a)];"),
 ("prolong w swap", "                        w *= use_other ? 1.0 : 3.0;\n                        if (cc[d] < 0 || cc[d] >= nc[d]) {", "                        w *= use_other ? 3.0 : 1.0;\n                        if (cc[d] < 0 || cc[d] >= nc[d]) {"),
 ("prolong side", "oth[d] = par[d] + ((c[d] % 2 == 0) ? -1 : 1);", "oth[d] = par[d] + ((c[d] % 2 == 0) ? 1 : -1);"),
 ("prolong /64", "s += (w / 64.0) * e[idx3(nc, cc[0], cc[1], cc[2])];", "s += (w / 27.0) * e[idx3(nc, cc[0], cc[1], cc[2])];"),
 ("prolong dirichlet", "                            if (dirichlet)\n                                valid = 0;", "                            if (0)\n                                valid = 0;"),
 ("levels >=4", "if (nx < 4 || nx % 2 != 0)", "if (nx < 2 || nx % 2 != 0)"),
 ("fas rhs sign", "C->f[c] = C->d[c] - rd[c];", "C->f[c] = C->d[c] + rd[c];"),
 ("corr sign", "e[c] = C->u[c] - C->uR[c];", "e[c] = C->uR[c] - C->u[c];"),
 ("restrict d of u", "restrict_avg(L->d, L->n, C->d);", "restrict_avg(L->u, L->n, C->d);"),
 ("coarse h", "        hh *= 2.0;\n", "        hh *= 1.0;\n"),
 ("coarse rho = 1", "restrict_avg(H->lev[l - 1].rho, H->lev[l - 1].n, L->rho);", "for (long c = 0; c < L->ncell; c++) L->rho[c] = 1.0;"),
 ("pinterp w", "            w *= use_other ? 1.0 : 3.0;\n            if (cc[d] < 0 || cc[d] >= np_[d]) {", "            w *= use_other ? 3.0 : 1.0;\n            if (cc[d] < 0 || cc[d] >= np_[d]) {"),
 ("pinterp side", "oth[d] = pc + ((fg - 2 * pc == 0) ? -1 : 1);", "oth[d] = pc + ((fg - 2 * pc == 0) ? 1 : -1);"),
 ("pinterp org", "int fg = 2 * org[d] + g[d];", "int fg = org[d] + g[d];"),
 ("ub mean", "ub_out[foff[f] + (long)Q * n[p] + P] = 0.5 * (ug + ui);", "ub_out[foff[f] + (long)Q * n[p] + P] = ug;"),
 ("ghost side", "ghost[ax] = (f % 2) ? n[ax] : -1;", "ghost[ax] = (f % 2) ? n[ax] - 1 : 0;"),
 ("cic shift", "double x = pos[3 * p + d] * n[d] - 0.5;", "double x = pos[3 * p + d] * n[d];"),
 ("cic weight", "w *= hi ? t[d] : (1.0 - t[d]);", "w *= hi ? (1.0 - t[d]) : t[d];"),
 ("cic mass", "double mass = (double)nc / (double)np;", "double mass = 1.0;"),
 ("face_axes", "*q = (ax == 2) ? 1 : 2;", "*q = (ax == 1) ? 1 : 2;"),
 ("face_value idx", "return L->ub[L->foff[f] + (long)c[q] * L->n[p] + c[p]];", "return L->ub[L->foff[f] + (long)c[p] * L->n[q] + c[q]];"),
]

EXPECTED_SURVIVORS = {"coarse rho = 1"}


def scratch_tree(w):
    if os.path.exists(w):
        shutil.rmtree(w)
    os.makedirs(w)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(w, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(w, "tests"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(w, "paper_1110_1379_gb300"))
    for f in ("__init__.py", "synth.py"):
        shutil.copy(os.path.join(ROOT, "paper_1110_1379_gb300", f),
                    os.path.join(w, "paper_1110_1379_gb300", f))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workdir", default=None, help="scratch folder (default: a temporary one)")
    ap.add_argument("names", nargs="*", help="run only these mutants")
    args = ap.parse_args()
    w = os.path.join(args.workdir or tempfile.mkdtemp(), "tree")
    scratch_tree(w)
    src = open(os.path.join(ROOT, "oracle", "fr_oracle.c")).read()
    survivors = []
    for name, a, b in MUTANTS:
        if args.names and name not in args.names:
            continue
        if src.count(a) != 1:
            print(f"STALE    {name}: the original text occurs {src.count(a)} times")
            survivors.append(name)
            continue
        with open(os.path.join(w, "oracle", "fr_oracle.c"), "w") as fh:
            fh.write(src.replace(a, b))
        shutil.rmtree(os.path.join(w, "oracle", "_build"), ignore_errors=True)
        t0 = time.time()
        r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                            "-m", "not gpu", "-p", "no:cacheprovider"], cwd=w,
                           capture_output=True, text=True)
        failed = [ln for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))]
        caught = r.returncode != 0
        if not caught:
            survivors.append(name)
        print(f"{'caught  ' if caught else 'SURVIVED'} {name:28s} {time.time() - t0:5.1f} s "
              f"{failed[0][:90] if failed else ''}", flush=True)
    unexpected = [n for n in survivors if n not in EXPECTED_SURVIVORS]
    print("survivors:", survivors, "unexpected:", unexpected)
    return 1 if unexpected else 0


if __name__ == "__main__":
    sys.exit(main())
