"""Planted mistakes: the oracle's pins must catch each of them.

Every case plants one plausible mistake -- a dropped term, a wrong sign, a
wrong index or operand, an off-by-one in the schedule -- in a copy of one of
the oracle's C sources, compiles the copy with the oracle's own flags, and
runs that source's pins (`test_oracle_pins.py` for fv_oracle.c,
`test_oracle_mlp.py` for mlp_oracle.c) in a child process that loads the
copy through FV_ORACLE_LIB.  A case passes when at least one pin fails.  The
unmodified oracle passes every pin (the pin files themselves).  CPU only:
the copies live in pytest's temporary directory.

Mistakes that leave every result unchanged (the sign of a Newton slope, say,
which changes only how the iteration converges) are not planted: no pin on
results can see them.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from oracle import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FV, MLP = B.SRCS

# (name, source, text, replacement, occurrence): `text` appears in the
# source; the occurrence-th appearance (0-based) is replaced.
MUTANTS = [
    # Riemann solver (Toro ch. 4)
    ("shock pressure function: sign of B", FV,
     "double q = sqrt(A / (p + B));", "double q = sqrt(A / (p - B));", 0),
    ("rarefaction pressure function: gamma+1 for gamma-1", FV,
     "*f = (2.0 * aK / G->gm1) * (pow(pr, z) - 1.0);",
     "*f = (2.0 * aK / G->gp1) * (pow(pr, z) - 1.0);", 0),
    ("Newton function: sign of du", FV,
     "double pn = p - (fL + fR + du) / (dfL + dfR);",
     "double pn = p - (fL + fR - du) / (dfL + dfR);", 0),
    ("star velocity: fL and fR swapped", FV,
     "*us = 0.5 * (uL + uR) + 0.5 * (fR - fL);", "*us = 0.5 * (uL + uR) + 0.5 * (fL - fR);", 0),
    ("two-rarefaction guess: sign of du", FV,
     "double num = aL + aR - 0.5 * G->gm1 * du;", "double num = aL + aR + 0.5 * G->gm1 * du;", 0),
    ("left shock star density: dropped k", FV,
     "*r = rL * ((q + k) / (k * q + 1.0));", "*r = rL * ((q + k) / (q + 1.0));", 0),
    ("right rarefaction fan: sign of the characteristic term", FV,
     "double c = 2.0 / gp1 - (gm1 / (gp1 * aR)) * (uR - xi);",
     "double c = 2.0 / gp1 + (gm1 / (gp1 * aR)) * (uR - xi);", 0),
    ("shock pressure function: gamma 1.4 hard-coded", FV,
     "double A = 2.0 / (G->gp1 * rK);", "double A = 2.0 / (2.4 * rK);", 0),
    ("left fan tail: gamma 1.4 hard-coded in the sound speed ratio", FV,
     "double asL = aL * pow(ps / pL, gm1 / (2.0 * g));", "double asL = aL * pow(ps / pL, 1.0 / 7.0);", 0),
    ("left star density behind a rarefaction: exponent gamma", FV,
     "*r = rL * pow(ps / pL, 1.0 / g);", "*r = rL * pow(ps / pL, g);", 0),
    # flux assembly
    ("tangential velocity from the downwind side", FV,
     "const double *Ws = side == 0 ? WL : WR;", "const double *Ws = side == 0 ? WR : WL;", 0),
    ("Godunov energy: gamma 1.4 hard-coded", FV,
     "double E0 = p0 / G->gm1 +", "double E0 = p0 / 0.4 +", 0),
    ("transmissive energy: gamma 1.4 hard-coded", FV,
     "double E = p / G->gm1 +", "double E = p / 0.4 +", 0),
    ("energy flux: dropped p", FV,
     "F[4] = un0 * (E0 + p0);", "F[4] = un0 * E0;", 0),
    ("momentum flux: dropped pressure", FV,
     "for (int d = 0; d < 3; ++d) F[1 + d] = mass * V0[d] + p0 * n[d];",
     "for (int d = 0; d < 3; ++d) F[1 + d] = mass * V0[d];", 0),
    ("wall flux: pressure of the unmirrored problem", FV,
     "int rc = riemann_star(G, WL[0], un, WL[4], WL[0], -un, WL[4], &ps, &us, iters);",
     "int rc = riemann_star(G, WL[0], un, WL[4], WL[0], un, WL[4], &ps, &us, iters);", 0),
    # primitives, ghost states, limiter
    ("kinetic energy without 1/2 (conserved to primitive)", FV,
     "double ke = 0.5 * r * ((u * u + v * v) + w * w);",
     "double ke = r * ((u * u + v * v) + w * w);", 0),
    ("internal energy p (gamma-1) (primitive to conserved)", FV,
     "U[4] = W[4] / G->gm1 + 0.5 * r", "U[4] = W[4] * G->gm1 + 0.5 * r", 0),
    ("wall ghost: normal velocity removed, not mirrored", FV,
     "for (int d = 0; d < 3; ++d) Wg[1 + d] = W[1 + d] - (2.0 * un) * n[d];",
     "for (int d = 0; d < 3; ++d) Wg[1 + d] = W[1 + d] - un * n[d];", 0),
    ("minmod picks the larger slope", FV,
     "if (a > 0.0 && b > 0.0) return a < b ? a : b;", "if (a > 0.0 && b > 0.0) return a > b ? a : b;", 0),
    ("minmod picks the larger slope when both are negative", FV,
     "if (a < 0.0 && b < 0.0) return a > b ? a : b;", "if (a < 0.0 && b < 0.0) return a < b ? a : b;", 0),
    ("MUSCL without the 1/2", FV,
     "WR[c] = Wj[c] - 0.5 * minmod(2.0 * gjr - dW, dW);", "WR[c] = Wj[c] - minmod(2.0 * gjr - dW, dW);", 0),
    ("MUSCL left state: sign of dW inside the limiter", FV,
     "WL[c] = Wi[c] + 0.5 * minmod(2.0 * gir - dW, dW);",
     "WL[c] = Wi[c] + 0.5 * minmod(2.0 * gir + dW, dW);", 0),
    ("MUSCL right state from the left cell's gradient", FV,
     "double gjr = (gj[3 * c] * r[0] + gj[3 * c + 1] * r[1]) + gj[3 * c + 2] * r[2];",
     "double gjr = (gi[3 * c] * r[0] + gi[3 * c + 1] * r[1]) + gi[3 * c + 2] * r[2];", 0),
    ("left shock speed: sign of the sound-speed term", FV,
     "double SL = uL - aL * sqrt(", "double SL = uL + aL * sqrt(", 0),
    # geometry and the least-squares gradient
    ("cell centroid: 1/5 for 1/4", FV,
     "+ x[3][d]) * 0.25;", "+ x[3][d]) * 0.2;", 0),
    ("face normals toward the owner", FV,
     "if (vdot(av, to) > 0.0)", "if (vdot(av, to) < 0.0)", 0),
    ("LS matrix inverse: sign of a cofactor", FV,
     "double c01 = M[1][2] * M[2][0] - M[1][0] * M[2][2];",
     "double c01 = M[1][0] * M[2][2] - M[1][2] * M[2][0];", 0),
    ("scheme gradient: weight components transposed", FV,
     "for (int a = 0; a < 3; ++a) g[3 * c + a] += w[a] * d;",
     "for (int a = 0; a < 3; ++a) g[3 * c + a] += w[2 - a] * d;", 0),
    ("face area without 1/2", FV,
     "for (int d = 0; d < 3; ++d) av[d] *= 0.5;", "for (int d = 0; d < 3; ++d) av[d] *= 1.0;", 0),
    ("ghost centroid at the face, not mirrored", FV,
     "double s = 2.0 * vdot(dl, o->fnrm + 3 * f);", "double s = vdot(dl, o->fnrm + 3 * f);", 0),
    # local step and levels (Alg. 2)
    ("local step without the factor 2", FV,
     "return (((2.0 * o->cfl) * o->vol[i]) * r) / S;", "return ((o->cfl * o->vol[i]) * r) / S;", 0),
    ("local step: c in place of rho c", FV,
     "double rc = sqrt((o->gas.g * p) * r);", "double rc = sqrt((o->gas.g * p) / r);", 0),
    ("local step: signed normal velocity", FV,
     "S = S + o->farea[f] * (fabs(mn) + rc);", "S = S + o->farea[f] * (mn + rc);", 0),
    ("neighbour rule allows a jump of two levels", FV,
     "if (o->lev[i] > o->lev[nb] + 1) {", "if (o->lev[i] > o->lev[nb] + 2) {", 0),
    ("face level = the coarser side", FV,
     "o->flev[f] = a < b ? a : b;", "o->flev[f] = a > b ? a : b;", 0),
    # schedule and time consistency
    ("tau(s) from s instead of s - 1", FV,
     "if (((s - 1) % (1 << tmp)) == 0) tau = tmp;", "if ((s % (1 << tmp)) == 0) tau = tmp;", 0),
    ("end set from s - 1", FV,
     "for (int k = 0; k <= theta && (s % (1 << k)) == 0; ++k) {",
     "for (int k = 0; k <= theta && ((s - 1) % (1 << k)) == 0; ++k) {", 0),
    ("interpolation weight reversed", FV,
     "double w = ldexp((double)num, -k);", "double w = 1.0 - ldexp((double)num, -k);", 0),
    # predictor, corrector, interfaces, ledger
    ("predictor: sign of the residual", FV,
     "double R = -S[c] / o->vol[i];", "double R = S[c] / o->vol[i];", 0),
    ("predictor step of the next level", FV,
     "double dtk = ldexp(o->dtmin, k);", "double dtk = ldexp(o->dtmin, k + 1);", 0),
    ("corrector: end-of-step flux only (dropped F1)", FV,
     "double phi = dtk * (0.5 * (o->F1A[5 * f + c] + F2A[c]));", "double phi = dtk * F2A[c];", 0),
    ("interface accumulator overwritten, not summed", FV,
     "if (interface) o->ACC[5 * f + c] += phi;", "if (interface) o->ACC[5 * f + c] = phi;", 0),
    ("interface accumulator never reset", FV,
     "for (int c = 0; c < 5; ++c) o->ACC[5 * f + c] = 0.0;", "for (int c = 0; c < 5; ++c) (void)0;", 0),
    ("boundary ledger misses the corrector integral", FV,
     "if (o->fnb[f] < 0) o->BND[5 * f + c] += phi;", "(void)0;", 0),
    ("global Heun step: dropped 1/2", FV,
     "double phi = dt * (0.5 * (o->F1A[5 * f + c] + F2A[c]));",
     "double phi = dt * (o->F1A[5 * f + c] + F2A[c]);", 0),
    ("boundary ledger misses the paper-order corrector integral", FV,
     "if (o->fnb[f] < 0) o->BND[5 * f + c] += phi;", "(void)0;", 1),
    ("residual: sign", FV,
     "for (int c = 0; c < 5; ++c) R_soa[c * o->nc + i] = -S[c] / o->vol[i];",
     "for (int c = 0; c < 5; ++c) R_soa[c * o->nc + i] = S[c] / o->vol[i];", 0),
    ("residual at stage 2 one subiteration after the step start", FV,
     "int64_t T = o->tn[k] + (stage == 2 ? ((int64_t)1 << k) : 0);",
     "int64_t T = o->tn[k] + (stage == 2 ? 1 : 0);", 0),
    ("global Heun step: second stage on U^n", FV,
     "  o->U = o->Us;\n  compute_W(o, 0);", "  compute_W(o, 0);", 0),
    ("face sign of the neighbour cell", FV,
     "o->csgn[4 * nb->tet + nb->j] = -1;", "o->csgn[4 * nb->tet + nb->j] = 1;", 0),
    ("LS weights: offsets of the neighbour's faces not reversed", FV,
     "double s = o->csgn[4 * i + j] > 0 ? 1.0 : -1.0;", "double s = 1.0;", 0),
    ("state check accepts a negative pressure", FV,
     "return (W[0] > 0.0 && W[4] > 0.0 && isfinite(W[0])",
     "return (W[0] > 0.0 && isfinite(W[0])", 0),
    ("predictor gradients only for the faces' owner cells", FV,
     "if (o->fnb[f] >= 0) o->mark[o->fnb[f]] = 1;", "(void)0;", 0),
    ("faces of the highest active level skipped at the step start", FV,
     "    if (o->flev[f] <= tau) {\n      o->mark", "    if (o->flev[f] < tau) {\n      o->mark", 0),
    # the paper's order
    ("paper order: no extrapolation past the predicted state", FV,
     "} else if (num == ((int64_t)1 << k)) {", "} else if (num >= ((int64_t)1 << k)) {", 0),
    ("paper order: commit also corrects own-level faces", FV,
     "if (o->flev[f] >= k) continue;", "if (o->flev[f] > k) continue;", 0),
    ("paper order: provisional integral with the corrector's sign", FV,
     "o->ACC[5 * f + c] -= prov;", "o->ACC[5 * f + c] += prov;", 0),
    ("paper order: provisional interface integral over half the step", FV,
     "double prov = dtk * o->F1A[5 * f + c];", "double prov = 0.5 * dtk * o->F1A[5 * f + c];", 0),
    ("paper order: commit ignores the interface correction", FV,
     "o->U[5 * i + c] = any ? o->Us[5 * i + c] - S[c] / o->vol[i] : o->Us[5 * i + c];",
     "o->U[5 * i + c] = o->Us[5 * i + c];", 0),
    ("paper order: commit keeps the interface accumulators", FV,
     "for (int c = 0; c < 5; ++c) o->ACC[5 * f + c] = 0.0;", "for (int c = 0; c < 5; ++c) (void)0;", 1),
    ("paper order: correctors finest first", FV,
     "for (int k = tau; k >= 0; --k) {\n      if (idx == 0) {\n        ph.kind = 2;",
     "for (int k = 0; k <= tau; ++k) {\n      if (idx == 0) {\n        ph.kind = 2;", 0),
    # the learned guess's reference (features, targets, network, training)
    ("GELU without 1/2", MLP,
     "return 0.5 * x * (1.0 + tanh(u));", "return x * (1.0 + tanh(u));", 0),
    ("GELU: sign of the cubic term", MLP,
     "double u = K_GELU * (x + C_GELU * x * x * x);", "double u = K_GELU * (x - C_GELU * x * x * x);", 0),
    ("GELU slope: 2 for 3 in the cubic's derivative", MLP,
     "double du = K_GELU * (1.0 + 3.0 * C_GELU * x * x);",
     "double du = K_GELU * (1.0 + 2.0 * C_GELU * x * x);", 0),
    ("feature: right pressure over the mean density", MLP,
     "x[5] = (pair[5] - pb) / pb;", "x[5] = (pair[5] - pb) / rb;", 0),
    ("two-rarefaction guess (learned-guess side): sign of du", MLP,
     "double num = aL + aR - 0.5 * (gamma - 1.0) * (uR - uL);",
     "double num = aL + aR + 0.5 * (gamma - 1.0) * (uR - uL);", 0),
    ("shock scale squared, not cubed", MLP, "return r * r * r;", "return r * r;", 0),
    ("feature: left velocity not taken relative to the mean", MLP,
     "x[1] = (pair[1] - ub) / ab;", "x[1] = pair[1] / ab;", 0),
    ("target 0 relative to the two-rarefaction guess", MLP,
     "if (target == 0) return log(ps / pb);", "if (target == 0) return log(ps / ptr);", 0),
    ("target 1: log of the inverse ratio", MLP,
     "return sc > 0.0 ? log(ps / ptr) / sc : 0.0;", "return sc > 0.0 ? log(ptr / ps) / sc : 0.0;", 0),
    ("forward pass: first layer transposed", MLP,
     "for (int i = 0; i < NIN; ++i) s += th[OFF_W1 + o * NIN + i] * x[i];",
     "for (int i = 0; i < NIN; ++i) s += th[OFF_W1 + i * H + o] * x[i];", 0),
    ("forward pass: second layer transposed", MLP,
     "for (int i = 0; i < H; ++i) s += th[OFF_W2 + o * H + i] * h1[i];",
     "for (int i = 0; i < H; ++i) s += th[OFF_W2 + i * H + o] * h1[i];", 0),
    ("backward pass: slope at the first layer's pre-activation", MLP,
     "d2[i] = dy * theta[OFF_W3 + i] * orc_gelu_grad(a2[i]);",
     "d2[i] = dy * theta[OFF_W3 + i] * orc_gelu_grad(a1[i]);", 0),
    ("backward pass: second layer not transposed", MLP,
     "for (int o = 0; o < H; ++o) s1 += theta[OFF_W2 + o * H + i] * d2[o];",
     "for (int o = 0; o < H; ++o) s1 += theta[OFF_W2 + i * H + o] * d2[o];", 0),
    ("loss gradient without the 2", MLP,
     "double dy = 2.0 * e / (double)n;", "double dy = e / (double)n;", 0),
    ("Adam without bias correction", MLP,
     "theta[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);",
     "theta[k] -= lr * m[k] / (sqrt(v[k]) + eps);", 0),
    ("bfloat16 rounding: ties away from zero", MLP,
     "u += 0x7fffu + ((u >> 16) & 1u);", "u += 0x8000u;", 0),
    ("mean sound speed from p rho instead of p / rho", MLP,
     "double ab = sqrt(gamma * pb / rb);", "double ab = sqrt(gamma * pb * rb);", 0),
    ("quantised pass: inputs not rounded", MLP,
     "xq[i] = (double)to_bf16(x[NIN * s + i]);", "xq[i] = (double)x[NIN * s + i];", 0),
    ("quantised pass: output weights rounded too", MLP,
     "out += (double)theta[OFF_W3 + o] * orc_gelu(a);",
     "out += (double)to_bf16(theta[OFF_W3 + o]) * orc_gelu(a);", 0),
    ("loss not averaged over the samples", MLP, "*loss = L / (double)n;", "*loss = L;", 0),
    ("Adam first moment with beta2", MLP,
     "m[k] = b1 * m[k] + (1.0 - b1) * grad[k];", "m[k] = b1 * m[k] + (1.0 - b2) * grad[k];", 0),
    ("quantised pass: first hidden layer not rounded", MLP,
     "h1[o] = (double)to_bf16((float)orc_gelu(a));", "h1[o] = orc_gelu(a);", 0),
]


def _read(path):
    with open(path) as fh:
        return fh.read()


def _plant(src, text, repl, occ):
    pos = -1
    for _ in range(occ + 1):
        pos = src.find(text, pos + 1)
        assert pos >= 0, text
    return src[:pos] + repl + src[pos + len(text):]


# the pins of each source file
PINS = {FV: "tests/test_oracle_pins.py", MLP: "tests/test_oracle_mlp.py"}


def _run_pins(lib, pins):
    env = dict(os.environ, FV_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", pins]
    try:
        r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return None, "timeout"
    return r.returncode, (r.stdout + r.stderr)[-600:]


def test_mutation_sites_are_unique_and_present():
    """Every planted text exists in the current source (a refactor that
    removes one must update its case)."""
    srcs = {FV: _read(FV), MLP: _read(MLP)}
    for name, path, text, repl, occ in MUTANTS:
        assert srcs[path].count(text) > occ, name
        assert text != repl, name


@pytest.mark.slow
def test_every_planted_mistake_fails_a_pin(tmp_path):
    srcs = {FV: _read(FV), MLP: _read(MLP)}

    def job(idx):
        name, path, text, repl, occ = MUTANTS[idx]
        d = tmp_path / f"m{idx}"
        d.mkdir()
        files = []
        for p in (FV, MLP):
            out = d / os.path.basename(p)
            out.write_text(_plant(srcs[p], text, repl, occ) if p == path else srcs[p])
            files.append(str(out))
        lib = B.compile_lib(files, str(d / "liboracle.so"))
        rc, tail = _run_pins(lib, PINS[path])
        return name, rc, tail

    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        results = list(ex.map(job, range(len(MUTANTS))))
    survivors = [(n, t) for n, rc, t in results if rc == 0]
    assert not survivors, "planted mistakes no pin caught:\n" + "\n".join(
        f"- {n}" for n, _ in survivors)
    # a planted mistake is caught by a failing pin, not by a hang
    assert all(rc is not None for _, rc, _ in results), [n for n, rc, _ in results if rc is None]
