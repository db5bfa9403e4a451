"""Mutation check of the oracle's pins (test infrastructure, not part of the
library).

Each entry plants one plausible mistake in an oracle file (``fr_oracle.c``,
``oracle.py``, ``symmetron.py``, ``masked.py``, ``poisson.py``, ``particles.py``: a wrong
constant, sign, index, weight or a dropped term) in a scratch copy of
``oracle/`` and ``tests/`` and runs that file's pin tests against it; a
mistake that no pin catches is reported as a survivor.  One survivor is
expected (``EXPECTED_SURVIVORS``): the f(R) coarse density set to 1, whose
terms cancel between L^H(u^H) and L^H(R u^h) in the FAS right-hand side
(Sec. V.B.2), so that mutant computes the same result.  Mistakes that change
only the iteration path (level rules, sweep order, clamps, coarse-level set-up)
are caught by pins that write those steps out by hand.

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

# (name, original text, mistaken text) per oracle file
MUT_C = [
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
 ("rms norm", "return n > 0 ? sqrt(s / (double)n) : 0.0;", "return n > 0 ? sqrt(s) : 0.0;"),
 ("cap clamp sign", "                    if (du > cap)\n                        du = cap;", "                    if (du > cap)\n                        du = -cap;"),
 ("residual drops f", "d[ci] = lv - (L->f ? L->f[ci] : 0.0);", "d[ci] = lv;"),
 ("pinterp no wrap", "cc[d] = ((cc[d] % np_[d]) + np_[d]) % np_[d];", "cc[d] = cc[d] < 0 ? 0 : np_[d] - 1;"),
 ("cic truncation", "double fl = floor(x);", "double fl = (double)(long)x;"),
 ("ngs black first", "                    if ((i + j + k) % 2 != colour)\n                        continue;\n                    long ci = idx3(L->n, i, j, k);\n                    double lv, dl;", "                    if ((i + j + k + 1) % 2 != colour)\n                        continue;\n                    long ci = idx3(L->n, i, j, k);\n                    double lv, dl;"),
 ("coarsest rule", "double thr = fmax(1e-3 * r0, 0.1 * H->tol);", "double thr = fmax(1e-1 * r0, 0.1 * H->tol);"),
 ("post count", "    for (int s = 0; s < H->post_sw; s++)\n        ngs_sweep(L, &H->m, H->cap);\n}", "    for (int s = 0; s < H->pre_sw; s++)\n        ngs_sweep(L, &H->m, H->cap);\n}"),
 ("face_value idx", "return L->ub[L->foff[f] + (long)c[q] * L->n[p] + c[p]];", "return L->ub[L->foff[f] + (long)c[p] * L->n[q] + c[q]];"),
]

MUT_SYMMETRON = [
 ("sy A factor 2", "A = 2.0 * lambda0 * lambda0 / (a * a * h * h)", "A = lambda0 * lambda0 / (a * a * h * h)"),
 ("sy s power", "    s = (a_ssb / a) ** 3\n    return A, s", "    s = (a_ssb / a) ** 2\n    return A, s"),
 ("sy background", "return float(np.sqrt(max(0.0, 1.0 - s)))", "return float(np.sqrt(max(0.0, 1.0 - s * s)))"),
 ("sy laplacian -6", "    out = -6.0 * chi\n", "    out = -4.0 * chi\n"),
 ("sy cubic sign", "return A * laplacian_sum(chi) - ((s * rho - 1.0) * chi + chi ** 3)", "return A * laplacian_sum(chi) - ((s * rho - 1.0) * chi - chi ** 3)"),
 ("sy mass sign", "return A * laplacian_sum(chi) - ((s * rho - 1.0) * chi + chi ** 3)", "return A * laplacian_sum(chi) - ((s * rho + 1.0) * chi + chi ** 3)"),
 ("sy deriv 3chi2", "return -6.0 * A - ((s * rho - 1.0) + 3.0 * chi * chi)", "return -6.0 * A - ((s * rho - 1.0) + chi * chi)"),
 ("sy deriv -6A", "return -6.0 * A - ((s * rho - 1.0) + 3.0 * chi * chi)", "return -4.0 * A - ((s * rho - 1.0) + 3.0 * chi * chi)"),
 ("sy newton sign", "d = -r / derivative(chi, rho, A, s)", "d = r / derivative(chi, rho, A, s)"),
 ("sy restrict", "return a.reshape(n2 // 2, 2, n1 // 2, 2, n0 // 2, 2).mean(axis=(1, 3, 5))", "return a.reshape(n2 // 2, 2, n1 // 2, 2, n0 // 2, 2).sum(axis=(1, 3, 5)) / 4.0"),
 ("sy prolong weights", "out = 0.75 * near + 0.25 * far", "out = 0.25 * near + 0.75 * far"),
 ("sy prolong side", "idx[ax] = slice(1, None, 2)", "idx[ax] = slice(0, None, 2)"),
 ("sy coarse A", "AH = 0.25 * A", "AH = 0.5 * A"),
 ("sy fas rhs sign", "fH = operator(uR, rhoH, AH, s) - restrict(d)", "fH = operator(uR, rhoH, AH, s) + restrict(d)"),
 ("sy correction sign", "chi = chi + prolong(uH - uR)", "chi = chi + prolong(uR - uH)"),
 ("sy levels >= 4", "while all(v % 2 == 0 and v // 2 >= 4 for v in n):", "while all(v % 2 == 0 and v // 2 >= 2 for v in n):"),
 ("sy cap clamp", "d = np.clip(d, -cap, cap)\n            chi[m] += d[m]", "d = np.clip(d, -cap, 0.5 * cap)\n            chi[m] += d[m]"),
 ("sy coarsest rule", "lim = max(1e-3 * r0, 0.1 * tol)", "lim = max(1e-1 * r0, 0.1 * tol)"),
 ("sy coarse rho injection", "rhoH = restrict(rho)", "rhoH = rho[::2, ::2, ::2]"),
]

MUT_MASKED = [
 ("ma ub from relation", "ub = (m * ug - mg * ut) / (m - mg)", "ub = (m * ug + mg * ut) / (m - mg)"),
 ("ma flux sign", "t_reg = (bi + bj) * (uj - ui)", "t_reg = (bi + bj) * (ui - uj)"),
 ("ma dflux bj", "d_reg = bi * (uj - ui) - (bi + bj)", "d_reg = bj * (uj - ui) - (bi + bj)"),
 ("ma ratio inverted", "r = np.where(L.act, mj / np.where(L.act, L.m, 1.0), 0.0)", "r = np.where(L.act, np.where(L.act, L.m, 1.0) / mj, 0.0)"),
 ("ma ghost sign", "ug = ub - r * ub + r * ui", "ug = ub + r * ub - r * ui"),
 ("ma ghost dflux", "d_gh = (bi + r * bg) * (ug - ui) + (bi + bg) * (r - 1.0)", "d_gh = (bi + bg) * (ug - ui) + (bi + bg) * (r - 1.0)"),
 ("ma ghost dflux2", "d_gh = (bi + r * bg) * (ug - ui) + (bi + bg) * (r - 1.0)", "d_gh = (bi + r * bg) * (ug - ui) + (bi + bg) * (r + 1.0)"),
 ("ma s exponent", "s = np.exp(-ui / 2.0)  # n = 1", "s = np.exp(-ui / 3.0)  # n = 1"),
 ("ma dens sign", "Lv = L.pre * flux - model.dens * (L.rho - 1.0) + model.src * s - model.bkg", "Lv = L.pre * flux + model.dens * (L.rho - 1.0) + model.src * s - model.bkg"),
 ("ma dL src", "dL = L.pre * dflux - model.src * s / 2.0", "dL = L.pre * dflux - model.src * s"),
 ("ma newton sign", "du = np.clip(-relax * (Lv - L.f) / dL, -cap, cap)", "du = np.clip(relax * (Lv - L.f) / dL, -cap, cap)"),
 ("ma restrict all children", "return restrict_mean(np.where(act, d, 0.0))", "return restrict_mean(d)"),
 ("ma prolong weights", "w = (0.25, 0.75)", "w = (0.75, 0.25)"),
 ("ma prolong side", "oz = (1 if cz else -1) if dz == 0 else 0", "oz = (-1 if cz else 1) if dz == 0 else 0"),
 ("ma prolong masked fine", "return np.where(fine_act, out, 0.0)", "return out"),
 ("ma coarse ghosts overwritten", "uR = np.where(C.act, restrict_mean(L.u), C.u)", "uR = restrict_mean(L.u)"),
 ("ma fas rhs sign", "C.f = np.where(C.act, LH - restrict_active(d, L.act), 0.0)", "C.f = np.where(C.act, LH + restrict_active(d, L.act), 0.0)"),
 ("ma coarse masks by injection", "u0, mm, rr, hh = restrict_mean(u0), restrict_mean(mm), restrict_mean(rr), 2 * hh", "u0, mm, rr, hh = restrict_mean(u0), mm[::2, ::2, ::2], restrict_mean(rr), 2 * hh"),
 ("ma coarse h", "u0, mm, rr, hh = restrict_mean(u0), restrict_mean(mm), restrict_mean(rr), 2 * hh", "u0, mm, rr, hh = restrict_mean(u0), restrict_mean(mm), restrict_mean(rr), hh"),
 ("ma colour order", "for colour in (0, 1):\n        Lv, dL = cell_terms(L, model)", "for colour in (1, 0):\n        Lv, dL = cell_terms(L, model)"),
 ("ma levels >= 4", "while all(s % 2 == 0 and s // 2 >= 4 for s in m.shape):", "while all(s % 2 == 0 and s // 2 >= 2 for s in m.shape):"),
]

MUT_POISSON = [
 ("po xi a^2", "dr = (n * a * a * m.xi) ** (1.0 / (n + 1.0))", "dr = (n * a * m.xi) ** (1.0 / (n + 1.0))"),
 ("po exponent", "np.exp(-ut / (n + 1.0))", "np.exp(-ut / n)"),
 ("po background 4OL", "- 3.0 * (a ** -3 + 4.0 * ol / omega_m)", "- 3.0 * (a ** -3 + 3.0 * ol / omega_m)"),
 ("po density factor 2", "return 2.0 * omega_m * a * (rho - 1.0) - omega_m * a ** 4 * dr / 6.0", "return 1.5 * omega_m * a * (rho - 1.0) - omega_m * a ** 4 * dr / 6.0"),
 ("po dR over 6", "return 2.0 * omega_m * a * (rho - 1.0) - omega_m * a ** 4 * dr / 6.0", "return 2.0 * omega_m * a * (rho - 1.0) - omega_m * a ** 4 * dr / 3.0"),
 ("po stencil -6", "    out = -6.0 * phi\n", "    out = -4.0 * phi\n"),
 ("po ghost rule", "nb[idx] = 2.0 * faces[2 * (2 - ax) + side] - phi[idx]", "nb[idx] = faces[2 * (2 - ax) + side]"),
 ("po ghost face index", "nb[idx] = 2.0 * faces[2 * (2 - ax) + side] - phi[idx]", "nb[idx] = 2.0 * faces[2 * ax + side] - phi[idx]"),
 ("po eigen 4", "e = -4.0 * np.sin(np.pi * k / n) ** 2 / (h * h)", "e = -2.0 * np.sin(np.pi * k / n) ** 2 / (h * h)"),
 ("po eigen pi", "e = -4.0 * np.sin(np.pi * k / n) ** 2 / (h * h)", "e = -4.0 * np.sin(2.0 * np.pi * k / n) ** 2 / (h * h)"),
 ("po patch diag", "diag[bl] -= 1.0", "diag[bl] -= 2.0"),
 ("po patch rhs", "rhs[bl] -= 2.0 * faces[2 * (2 - ax) + side][..., :] * np.ones_like(rhs[bl])", "rhs[bl] -= faces[2 * (2 - ax) + side][..., :] * np.ones_like(rhs[bl])"),
]

MUT_PARTICLES = [
 ("pa centre offset", "x = pos[:, d] * n[d] - 0.5", "x = pos[:, d] * n[d]"),
 ("pa cic weights", "w = np.stack([1.0 - t, t], axis=1)", "w = np.stack([t, 1.0 - t], axis=1)"),
 ("pa tsc nearest", "c = np.floor(x + 0.5)", "c = np.floor(x)"),
 ("pa tsc centre weight", "0.75 - dd ** 2", "0.75 - 0.5 * dd ** 2"),
 ("pa tsc side weights", "w = np.stack([0.5 * (0.5 - dd) ** 2, 0.75 - dd ** 2, 0.5 * (0.5 + dd) ** 2], axis=1)", "w = np.stack([0.5 * (0.5 + dd) ** 2, 0.75 - dd ** 2, 0.5 * (0.5 - dd) ** 2], axis=1)"),
 ("pa mass", "mass = float(np.prod(shape)) / npart", "mass = 1.0"),
 ("pa axes swapped", "np.add.at(rho, (iz[:, c], iy[:, b], ix[:, a]), mass * wx[:, a] * wy[:, b] * wz[:, c])", "np.add.at(rho, (ix[:, a], iy[:, b], iz[:, c]), mass * wx[:, a] * wy[:, b] * wz[:, c])"),
 ("pa gradient sign", "gx = (np.roll(phi, -1, axis=2) - np.roll(phi, 1, axis=2)) * (n0 / 2.0)", "gx = (np.roll(phi, 1, axis=2) - np.roll(phi, -1, axis=2)) * (n0 / 2.0)"),
 ("pa gradient scale", "gy = (np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)) * (n1 / 2.0)", "gy = (np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1)) * n1"),
 ("pa force sign", "out[:, d] -= w * g[d][iz[:, c], iy[:, b], ix[:, a]]", "out[:, d] += w * g[d][iz[:, c], iy[:, b], ix[:, a]]"),
]

MUT_ORACLE_PY = [
 ("tau coarse h", "return (residual(restrict(u), restrict(rho), h=2.0 * h, **P)", "return (residual(restrict(u), restrict(rho), h=h, **P)"),
 ("tau sign", "            - restrict(residual(u, rho, h=h, **P)))", "            + restrict(residual(u, rho, h=h, **P)))"),
 ("tau coarse rho", "return (residual(restrict(u), restrict(rho), h=2.0 * h, **P)", "return (residual(restrict(u), rho[::2, ::2, ::2], h=2.0 * h, **P)"),
 ("levels patch h", "max_cycles=max_cycles, pre=pre, post=post, cap=cap, u0=u0, h=hp / 2.0,", "max_cycles=max_cycles, pre=pre, post=post, cap=cap, u0=u0, h=hp,"),
 ("levels parent", "up, periodic, hp = out[p[\"parent\"]].u, False, hs[p[\"parent\"]]", "up, periodic, hp = dom.u, False, hs[p[\"parent\"]]"),
 ("levels patch rho", "r = solve(p[\"rho\"], box=box,", "r = solve(np.ones_like(p[\"rho\"]), box=box,"),
]

# oracle file -> (pin tests, mutants)
TARGETS = {
    "fr_oracle.c": (["tests/test_oracle_pins.py"], MUT_C),
    "oracle.py": (["tests/test_oracle_pins.py"], MUT_ORACLE_PY),
    "symmetron.py": (["tests/test_symmetron_pins.py"], MUT_SYMMETRON),
    "masked.py": (["tests/test_mask_pins.py"], MUT_MASKED),
    "poisson.py": (["tests/test_poisson_pins.py"], MUT_POISSON),
    "particles.py": (["tests/test_particle_pins.py"], MUT_PARTICLES),
}

# survivors that no result can expose, with the reason
EXPECTED_SURVIVORS = {
    # equivalent: the coarse density terms cancel in the FAS right-hand side
    "coarse rho = 1",
}


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
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    survivors = []
    total = 0
    for fname, (tests, mutants) in TARGETS.items():
        path = os.path.join(w, "oracle", fname)
        src = open(os.path.join(ROOT, "oracle", fname)).read()
        for name, a, b in mutants:
            if args.names and name not in args.names:
                continue
            total += 1
            if src.count(a) != 1:
                print(f"STALE    {name}: the original text occurs {src.count(a)} times")
                survivors.append(name)
                continue
            with open(path, "w") as fh:
                fh.write(src.replace(a, b))
            shutil.rmtree(os.path.join(w, "oracle", "_build"), ignore_errors=True)
            t0 = time.time()
            r = subprocess.run([sys.executable, "-m", "pytest", *tests, "-x", "-q", "-m", "not gpu",
                                "-p", "no:cacheprovider"], cwd=w, env=env,
                               capture_output=True, text=True)
            failed = [ln for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))]
            caught = r.returncode != 0
            if not caught:
                survivors.append(name)
            print(f"{'caught  ' if caught else 'SURVIVED'} {fname:13s} {name:28s} "
                  f"{time.time() - t0:5.1f} s {failed[0][:80] if failed else ''}", flush=True)
        with open(path, "w") as fh:
            fh.write(src)
    print(f"{total} mutants")
    unexpected = [n for n in survivors if n not in EXPECTED_SURVIVORS]
    print("survivors:", survivors, "unexpected:", unexpected)
    return 1 if unexpected else 0


if __name__ == "__main__":
    sys.exit(main())
