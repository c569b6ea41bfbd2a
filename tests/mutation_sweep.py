"""Mutation sweep of the oracle's pins (run by hand; pytest does not collect it).

Each entry plants one plausible mistake (a sign, a dropped term, an index, a
weight, a constant) in a copy of oracle/grmhd_oracle.cpp, builds that copy in
a temporary folder and runs tests/test_oracle_pins.py against it through
ORACLE_SRC / ORACLE_BUILD.  A mistake that no pin catches is reported, and
the script exits 1 if any survives, apart from the equivalent mutants listed
in EQUIVALENT (mistakes that cannot change any result).

    python tests/mutation_sweep.py            # all mistakes, a few minutes
    python tests/mutation_sweep.py -k WENO    # those whose name contains WENO
"""
import argparse
import os
import shutil
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "grmhd_oracle.cpp")

# (name, original text, planted mistake); every original occurs once in SRC
MUTATIONS = [
    ('shift sign in vhat',
     'vh[i] = v[i] - beta[i] / alpha;',
     'vh[i] = v[i] + beta[i] / alpha;'),
    ('drop b_i in S flux',
     'o.F[1 + i] = alpha * o.U[1 + i] * vh[d] - alpha * bl[i] * Bt[d] / W;',
     'o.F[1 + i] = alpha * o.U[1 + i] * vh[d];'),
    ('Ptot uses b2 not b2/2',
     'real Ptot = P + 0.5 * b2;\n  // b_i',
     'real Ptot = P + b2;\n  // b_i'),
    ('RK3 weight',
     '{0.75, 0.25, 0.25}',
     '{0.75, 0.25, 0.3}'),
    ('WENO d1',
     'real a1 = 0.6 *',
     'real a1 = 0.5 *'),
    ('CT upwind swap',
     'if (fD > 0.0) return lowv;\n  if (fD < 0.0) return highv;',
     'if (fD > 0.0) return highv;\n  if (fD < 0.0) return lowv;'),
    ('drop dbeta source',
     'Gs[1 + a] = 0.5 * alpha * t + s2 - E * dal[a];',
     'Gs[1 + a] = 0.5 * alpha * t - E * dal[a];'),
    ('Gtau sign',
     'Gs[4] = alpha * kt - sd;',
     'Gs[4] = alpha * kt + sd;'),
    ('metric inverse index',
     'gi[4] = (g[1] * g[2] - g[0] * g[4]) / det;',
     'gi[4] = (g[1] * g[2] - g[0] * g[3]) / det;'),
    ('qbar sign',
     'e.qbar = s.q - 0.5 * s.b2 - 0.5',
     'e.qbar = s.q + 0.5 * s.b2 - 0.5'),
    ('face interp weight',
     '(-a + 9.0 * bq + 9.0 * cq - dq) / 16.0',
     '(-a + 9.0 * bq + 9.0 * cq - dq) / 15.0'),
    ('tau drops B2/W2',
     'out[4] = sdet * (rhohW2 + B2 - P - 0.5 * (Bv * Bv + B2 / (W * W)) - D);',
     'out[4] = sdet * (rhohW2 + B2 - P - 0.5 * (Bv * Bv) - D);'),
    ('DMP lower bound',
     'real lo = mn > 0.0 ? mn / M : mn * M;',
     'real lo = mn > 0.0 ? mn * M : mn / M;'),
    ('fofc both cells',
     'if (!(a || bb)) continue;',
     'if (!(a && bb)) continue;'),
    ('curl sign bf1',
     'curl = (real(emf[2][G.e(2, k, j + 1, i)]) - real(emf[2][G.e(2, k, j, i)])) / dx[1] -',
     'curl = (real(emf[2][G.e(2, k, j + 1, i)]) - real(emf[2][G.e(2, k, j, i)])) / dx[1] +'),
    ('HLLE diffusion sign',
     '+ lL * lR * (R.U[c] - L.U[c])',
     '- lL * lR * (R.U[c] - L.U[c])'),
    ('hyb K continuity exponent',
     'const real Kn = K * pow_(rb, Gj - Gn);',
     'const real Kn = K * pow_(rb, Gn - Gj);'),
    ('hyb a continuity drops Kn',
     'a = a + K * pow_(rb, Gj - 1.0) / (Gj - 1.0) - Kn * pow_(rb, Gn - 1.0) / (Gn - 1.0);',
     'a = a + K * pow_(rb, Gj - 1.0) / (Gj - 1.0);'),
    ('hyb cold eps index',
     'epsc = a + K * pow_(rho, Gi - 1.0) / (Gi - 1.0);',
     'epsc = a + K * pow_(rho, Gi - 1.0) / Gi;'),
    ('hyb eps thermal factor',
     'return epsc + (P - Pc) / ((eos_gth(p) - 1.0) * rho);',
     'return epsc + (P - Pc) / (eos_gth(p) * rho);'),
    ('hyb press thermal factor',
     'return Pc + (eos_gth(p) - 1.0) * rho * (eps - epsc);',
     'return Pc + eos_gth(p) * rho * (eps - epsc);'),
    ('hyb h drops P/rho',
     'return 1.0 + eos_eps(p, rho, P) + P / rho;',
     'return 1.0 + eos_eps(p, rho, P);'),
    ('hyb chi drops cold index',
     'return Gi * Pc + eos_gth(p) * (P - Pc);',
     'return eos_gth(p) * P;'),
    ('hyb pfloor drops Pc',
     'return Pc + rho * p.T_atm;',
     'return rho * p.T_atm;'),
    ('hyb epsmin factor',
     'return epsc + p.T_atm / (eos_gth(p) - 1.0);',
     'return epsc + p.T_atm;'),
    ('hyb krp eps_min ideal',
     'e.eps_min = s.hyb ? eos_epsmin(*s.hyb, e.rhohat) : s.eps_min;',
     'e.eps_min = s.eps_min;'),
    ('krp nu drops nuB',
     'real nu = max_(nuA, nuB);',
     'real nu = nuA;'),
    ('krp What from v2 not vhat2',
     'e.What = 1.0 / sqrt_(1.0 - e.vhat2);',
     'e.What = 1.0 / sqrt_(1.0 - 0.99 * e.vhat2);'),
    ('PLM vl factor',
     'return pr > 0.0 ? 2.0 * pr / (dl + dr) : real(0.0);',
     'return pr > 0.0 ? pr / (dl + dr) : real(0.0);'),
    ('PPM4 interface slope sign',
     'real aL = a[1] + 0.5 * (a[2] - a[1]) - (s1 - s0) / 6.0;',
     'real aL = a[1] + 0.5 * (a[2] - a[1]) + (s1 - s0) / 6.0;'),
    ('PPM4 overshoot factor',
     '      aL = 3.0 * aj - 2.0 * aR;\n    } else if',
     '      aL = 2.0 * aj - aR;\n    } else if'),
    ('PPM4 slope cap',
     'real m = min_(abs_(dc), min_(2.0 * abs_(dl), 2.0 * abs_(dr)));',
     'real m = min_(abs_(dc), min_(abs_(dl), abs_(dr)));'),
    ('PPMX face weight',
     'real f = 7.0 / 12.0 * (a0 + ap) - 1.0 / 12.0 * (am + app);',
     'real f = 7.0 / 12.0 * (a0 + ap) - 1.0 / 6.0 * (am + app);'),
    ('PPMX d2lim C',
     '  const real C = 1.25;\n  if (d > 0.0 && d1 > 0.0',
     '  const real C = 1.5;\n  if (d > 0.0 && d1 > 0.0'),
    ('PPMX overshoot factor',
     'if (abs_(dR) >= 2.0 * abs_(dL)) aR = aj - 2.0 * dL;',
     'if (abs_(dR) >= 2.0 * abs_(dL)) aR = aj - dL;'),
    ('LLF speed set',
     'real a = max_(max_(abs_(L.lm), abs_(L.lp)), max_(abs_(R.lm), abs_(R.lp)));',
     'real a = max_(abs_(L.lm), abs_(R.lp));'),
    ('LLF diffusion half',
     'F[c] = 0.5 * (L.F[c] + R.F[c]) - 0.5 * a * (R.U[c] - L.U[c]);',
     'F[c] = 0.5 * (L.F[c] + R.F[c]) - a * (R.U[c] - L.U[c]);'),
    ('HLLE lL no zero clamp',
     'real lL = min_(min_(L.lm, R.lm), real(0.0));',
     'real lL = min_(L.lm, R.lm);'),
    ('excision ignored',
     'const bool excise = p.alpha_exc > 0.0 && alpha < p.alpha_exc;',
     'const bool excise = false;'),
    ('sigma floor inverted',
     'D = B2 / p.sigma_max;',
     'D = B2 * p.sigma_max;'),
    ('tau_atm drops B2',
     'real tau_atm = D * eps_atm + 0.5 * B2;',
     'real tau_atm = D * eps_atm;'),
    ('D floor tau drops B2',
     'tau = D * eps_atm_rho + 0.5 * B2;',
     'tau = D * eps_atm_rho;'),
    ('WENO b2 weight',
     'real b2 = 13.0 / 12.0 * t * t + 0.25 * u * u;',
     'real b2 = 13.0 / 12.0 * t * t + 0.5 * u * u;'),
    ('WENO q1 stencil',
     'real q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;',
     'real q1 = (-b + 6.0 * c + d) / 6.0;'),
    ('WENO tau5',
     'real tau5 = abs_(b0 - b2);',
     'real tau5 = abs_(b0 - b1);'),
    ('S^ij drops Ptot gamma^ij',
     'Sij[sym(a, bq)] = sdet * (e * v[a] * v[bq] + Ptot * gi[sym(a, bq)] - bb[a] * bb[bq]);',
     'Sij[sym(a, bq)] = sdet * (e * v[a] * v[bq] - bb[a] * bb[bq]);'),
    ('S^ij bbar sign',
     'Sij[sym(a, bq)] = sdet * (e * v[a] * v[bq] + Ptot * gi[sym(a, bq)] - bb[a] * bb[bq]);',
     'Sij[sym(a, bq)] = sdet * (e * v[a] * v[bq] + Ptot * gi[sym(a, bq)] + bb[a] * bb[bq]);'),
    ('bbar drops W Bv v',
     'bb[a] = B[a] / W + W * Bv * v[a];',
     'bb[a] = B[a] / W;'),
    ('Gtau drops K S',
     'Gs[4] = alpha * kt - sd;',
     'Gs[4] = - sd;'),
    ('source E uses tau only',
     'real E = real(C.b->cons[4 * G.ncell + c]) + real(C.b->cons[0 * G.ncell + c]);',
     'real E = real(C.b->cons[4 * G.ncell + c]);'),
    ('source dgamma half',
     'Gs[1 + a] = 0.5 * alpha * t + s2 - E * dal[a];',
     'Gs[1 + a] = alpha * t + s2 - E * dal[a];'),
    ('source Su not raised',
     'sd = sd + Su[a] * dal[a];',
     'sd = sd + Sl[a] * dal[a];'),
    ('ecc sign',
     'ecc[0 * G.ncell + c] = val(-alpha * (vh[1] * B[2] - vh[2] * B[1]));',
     'ecc[0 * G.ncell + c] = val(alpha * (vh[1] * B[2] - vh[2] * B[1]));'),
    ('ecc z component index',
     'ecc[2 * G.ncell + c] = val(-alpha * (vh[0] * B[1] - vh[1] * B[0]));',
     'ecc[2 * G.ncell + c] = val(-alpha * (vh[0] * B[2] - vh[2] * B[0]));'),
    ('DMP upper bound',
     'real hi = mx > 0.0 ? mx * M : mx / M;',
     'real hi = mx > 0.0 ? mx / M : mx * M;'),
    ('RK2 second weight',
     'static const double RK2_W[2][3] = {{0.0, 1.0, 1.0}, {0.5, 0.5, 0.5}};',
     'static const double RK2_W[2][3] = {{0.0, 1.0, 1.0}, {0.5, 0.5, 1.0}};'),
    ('face floor threshold',
     '  if (s[0] < p.f_thr * p.rho_atm) {\n    s[0] = p.rho_atm;',
     '  if (s[0] < p.rho_atm) {\n    s[0] = p.rho_atm;'),
    ('vcap no rescale',
     'if (e.vcap) vs = sqrt_(s.vmax2 / (mu * mu * e.rbar2));',
     'if (e.vcap) vs = 1.0;'),
    ('source dal centred factor',
     'real inv2dx = 1.0 / (2.0 * C.b->dx[a]);',
     'real inv2dx = 1.0 / C.b->dx[a];'),
    ('b2 drops Bv^2',
     'real b2 = B2 / (W * W) + Bv * Bv;\n  real h = eos_h(C.p, rho, P);',
     'real b2 = B2 / (W * W);\n  real h = eos_h(C.p, rho, P);'),
    ('curl x-face drops dAy/dz',
     '                                    (Ay[G.e(1, k + 1, j, i)] - Ay[G.e(1, k, j, i)]) / dx[2];',
     '                                    (Ay[G.e(1, k + 1, j, i)] - Ay[G.e(1, k, j, i)]) / dx[2] * 0.0;'),
    ('curl z-face spacing',
     '        b->bf[2][G.f(2, k, j, i)] = (Ay[G.e(1, k, j, i + 1)] - Ay[G.e(1, k, j, i)]) / dx[0] -',
     '        b->bf[2][G.f(2, k, j, i)] = (Ay[G.e(1, k, j, i + 1)] - Ay[G.e(1, k, j, i)]) / dx[1] -'),
    ('bcc y average index',
     'C.b->bcc[1 * G.ncell + c] = val(0.5 * (real(C.b->bf[1][G.f(1, k, j, i)]) + real(C.b->bf[1][G.f(1, k, j + 1, i)])));',
     'C.b->bcc[1 * G.ncell + c] = val(0.5 * (real(C.b->bf[1][G.f(1, k, j, i)]) + real(C.b->bf[1][G.f(1, k, j, i)])));'),
    ('illinois final regula falsi',
     '  return a - fa * (b - a) / (fb - fa);\n}',
     '  return 0.5 * (a + b);\n}'),
    ('illinois no halving',
     '      if (side == -1) Fb = 0.5 * Fb;',
     '      if (side == -1) Fb = 1.0 * Fb;'),
    ('bracket no [mu+, 1] fallback',
     '    if (e1.f < 0.0) {\n      a = b; e0 = e1;\n      b = 1.0;',
     '    if (false) {\n      a = b; e0 = e1;\n      b = 1.0;'),
    ('krp rb2 not squared',
     '    s.rb2 = s.rb * s.rb;',
     '    s.rb2 = s.rb;'),
    ('krp b2 not per D',
     '    s.b2 = B2 / D;',
     '    s.b2 = B2;'),
    ('fofc fix keeps high order',
     '    reconstruct(donor ? 0 : C.p.recon, q, &L[v], &R[v]);',
     '    reconstruct(C.p.recon, q, &L[v], &R[v]);'),
    ('post-solve rho floor removed',
     '      if (rho < p.f_thr * rho_atm) {\n        rho = rho_atm;',
     '      if (false) {\n        rho = rho_atm;'),
    ('post-solve P floor removed',
     '        if (P < Pf) {\n          P = Pf;',
     '        if (false) {\n          P = Pf;'),
    ('stage 0 keeps no U^n',
     '          if (first) C.b->cons0[v * G.ncell + c] = C.b->cons[v * G.ncell + c];',
     '          if (false) C.b->cons0[v * G.ncell + c] = C.b->cons[v * G.ncell + c];'),
    ('p2c D without W',
     'real D = rho * W;\n  out[0]',
     'real D = rho;\n  out[0]'),
    ('p2c S drops Bv B_i',
     'out[1 + i] = sdet * ((rhohW2 + B2) * vl[i] - Bv * Bl[i]);',
     'out[1 + i] = sdet * ((rhohW2 + B2) * vl[i]);'),
    ('p2c tau keeps D',
     '- D);',
     ');'),
    ('metric det middle sign',
     '- g[1] * (g[1] * g[5] - g[4] * g[2])',
     '+ g[1] * (g[1] * g[5] - g[4] * g[2])'),
    ('metric lower y index',
     'out[1] = g[1] * in[0] + g[3] * in[1] + g[4] * in[2];',
     'out[1] = g[1] * in[0] + g[3] * in[1] + g[2] * in[2];'),
    ('krp rbar2 (1+x) factor',
     'mu * e.x * (1.0 + e.x) * s.rb2;',
     'mu * e.x * 2.0 * s.rb2;'),
    ('krp qbar perp sign',
     '- 0.5 * mu * mu * e.x * e.x * s.rperp2;',
     '+ 0.5 * mu * mu * e.x * e.x * s.rperp2;'),
    ('krp eps_raw drops v^2 W^2 term',
     '+ e.vhat2 * e.What * e.What / (1.0 + e.What);',
     ';'),
    ('krp nuA drops 1/W',
     '(1.0 + ahat) * (1.0 + e.eps) / e.What;',
     '(1.0 + ahat) * (1.0 + e.eps);'),
    ('krp rhohat times W',
     'e.rhohat = s.D / e.What;',
     'e.rhohat = s.D * e.What;'),
    ('flux divergence sign',
     'r = r - (fp - fm) / C.b->dx[d];',
     'r = r + (fp - fm) / C.b->dx[d];'),
    ('face B update sign',
     'bnew = bnew - bdt * curl;',
     'bnew = bnew + bdt * curl;'),
    ('CT upwind tie takes one side',
     'return 0.5 * (lowv + highv);',
     'return lowv;'),
    ('CT a-derivative weight',
     '+ 0.25 * (dEa_tq - dEa_q);',
     '+ 0.5 * (dEa_tq - dEa_q);'),
    ('CT b-derivative operand order',
     'real dEb_tq = upwind(f[1], Ebf_Am - E_AmBm, Ebf_A - E_ABm);',
     'real dEb_tq = upwind(f[1], Ebf_A - E_ABm, Ebf_Am - E_AmBm);'),
    ('mu_plus start from r^2',
     'real rpar2 = s.b2 > 0.0 ? s.rb2 / s.b2 : s.r2;',
     'real rpar2 = s.r2;'),
]

# nu = max(nu_A, nu_B) in the master function: with eps_raw as defined and
# vhat^2 What^2 = What^2 - 1, nu_B = (1 + ahat)(1 + eps_raw)/What, while nu_A
# uses epshat = max(eps_raw, eps_min) >= eps_raw; so nu_A >= nu_B for this
# EOS (no upper eps limit), also under the speed cap.
EQUIVALENT = {"krp nu drops nuB"}


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("-k", default="", help="only the mistakes whose name contains this")
    args = ap.parse_args()
    orig = open(SRC).read()
    survivors = []
    for name, a, b in MUTATIONS:
        if args.k not in name:
            continue
        if orig.count(a) != 1:
            print(f"{name:30s} anchor not found once", flush=True)
            survivors.append(name)
            continue
        tmp = tempfile.mkdtemp(prefix="oracle_mut_")
        try:
            src = os.path.join(tmp, "grmhd_oracle.cpp")
            with open(src, "w") as f:
                f.write(orig.replace(a, b))
            env = dict(os.environ, ORACLE_SRC=src, ORACLE_BUILD=os.path.join(tmp, "_build"))
            r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                                "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True)
            last = (r.stdout.strip().splitlines() or ["(no output)"])[-1]
            caught = r.returncode != 0
        finally:
            shutil.rmtree(tmp, ignore_errors=True)
        tag = "caught" if caught else ("equivalent" if name in EQUIVALENT else "SURVIVED")
        print(f"{name:30s} {tag:10s} {last}", flush=True)
        if not caught and name not in EQUIVALENT:
            survivors.append(name)
    if survivors:
        print("survivors:", ", ".join(survivors))
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
