"""The oracle's pins against planted mistakes: each case below alters one
line of a copy of the oracle (a dropped term, a flipped sign, a wrong index
or weight, a missing species or field) and the pins of the matching file
must fail on the altered copy.  The C oracle is rebuilt per case in a
temporary directory and loaded by the pin files in a subprocess (through
ORACLE_LIB); the beam-push oracle is re-executed from altered source in
process.  The copies and the planted mistakes live only in the temporary
directory; the oracle itself is never changed.

The axis readings (the AB2 history negated with rho and u_r when a ring
is reflected; an RK4 stage below the axis evaluated mirrored) are pinned
by the convergence order of a light ring's orbit through the axis against
an independent integration (tests/axis_orbit.py); their planted mistakes
are listed with the others."""
import concurrent.futures
import importlib.util
import os
import shutil
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (name, pin file, original text, planted text); each original occurs once
C_CASES = [
    # steps a3-a8 and the AB2 push of orc_run / slice_core
    ("B_drops_beam_term", "test_oracle_pins.py",
     "+ wr * s->bb[i] / pb\n                  + (w / (r * r))", "+ (w / (r * r))"),
    ("B_drops_u2_over_r2", "test_oracle_pins.py",
     "+ wr * s->bb[i] / pb\n                  + (w / (r * r)) * u * u / (pb * pb)", "+ wr * s->bb[i] / pb"),
    ("B_drops_u2_dpr", "test_oracle_pins.py",
     "+ (w / (r * r)) * u * u / (pb * pb)\n                  + wr * u * u * dpr / (pb * pb * pb)",
     "+ (w / (r * r)) * u * u / (pb * pb)"),
    ("B_flips_dzeta_term", "test_oracle_pins.py",
     "+ wr * u * u * dpr / (pb * pb * pb)\n                  - wr * u * dpz / (pb * pb);",
     "+ wr * u * u * dpr / (pb * pb * pb)\n                  + wr * u * dpz / (pb * pb);"),
    ("C_flips_one", "test_oracle_pins.py",
     "s->C[i] = -wr * (g / pb - 1.0 - u * u / (pb * pb));", "s->C[i] = -wr * (g / pb + 1.0 - u * u / (pb * pb));"),
    ("C_drops_u2", "test_oracle_pins.py",
     "s->C[i] = -wr * (g / pb - 1.0 - u * u / (pb * pb));", "s->C[i] = -wr * (g / pb - 1.0);"),
    ("A_extra_psibar", "test_oracle_pins.py", "s->A[i] = wr / pb;", "s->A[i] = wr / (pb * pb);"),
    ("dpr_drops_self_weight", "test_oracle_pins.py",
     "s->dpr[i] = (s->S[i] + s->wh[i] - ion_enclosed(r, dens, rho_max)) / r;",
     "s->dpr[i] = (s->S[i] - ion_enclosed(r, dens, rho_max)) / r;"),
    ("psi_drops_S_log", "test_oracle_pins.py",
     "s->psi[i] = (s->Ltot - s->L[i]) + s->S[i] * log(r) + ion_psi(r, dens, rho_max);",
     "s->psi[i] = (s->Ltot - s->L[i]) + ion_psi(r, dens, rho_max);"),
    ("dzeta_self_weight_inverted", "test_oracle_pins.py",
     "return -(suffix_above + (1.0 - wh_self / w_self) * t_self);", "return -(suffix_above + (wh_self / w_self) * t_self);"),
    ("dzeta_printed_sign", "test_oracle_pins.py",
     "return -(suffix_above + (1.0 - wh_self / w_self) * t_self);", "return (suffix_above + (1.0 - wh_self / w_self) * t_self);"),
    ("ion_psi_factor", "test_oracle_pins.py",
     "return 0.25 * n * (rho_max * rho_max - rho * rho) - q * log(rho_max);",
     "return 0.5 * n * (rho_max * rho_max - rho * rho) - q * log(rho_max);"),
    ("ion_column_unbounded", "test_oracle_pins.py", "double c = rho < rho_max ? rho : rho_max;", "double c = rho;"),
    ("gamma_sign", "test_oracle_pins.py",
     "s->gam[i] = (1.0 + u * u + pb * pb) / (2.0 * pb);", "s->gam[i] = (1.0 - u * u + pb * pb) / (2.0 * pb);"),
    ("t_without_psibar", "test_oracle_pins.py", "s->t[i] = s->w[i] * u / (r * pb);", "s->t[i] = s->w[i] * u / r;"),
    ("bp_one_sided_at_ring", "test_oracle_pins.py",
     "s->bp[i] = 0.5 * ((s->a[i] + s->a[i + 1]) * r + (s->b[i] + s->b[i + 1]) / r);",
     "s->bp[i] = s->a[i] * r + s->b[i] / r;"),
    ("self_weight_eighth", "test_oracle_pins.py",
     "if (what) what[j] = density * (0.5 * c * d - 0.125 * d * d);",
     "if (what) what[j] = density * (0.5 * c * d - 0.25 * d * d);"),
    ("beam_count_inclusive", "test_oracle_pins.py",
     "double Q = bs->P[lower_bound(bs->r, bs->m, rho)];",
     "double Q = bs->P[lower_bound(bs->r, bs->m, rho) < bs->m ? lower_bound(bs->r, bs->m, rho) + 1 : bs->m];"),
    ("push_force_sign", "test_oracle_pins.py",
     "double fu = s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]);",
     "double fu = s.gam[i] * s.dpr[i] / pb + (s.bp[i] + s.bb[i]);"),
    ("push_drops_beam_field", "test_oracle_pins.py",
     "double fu = s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]);", "double fu = s.gam[i] * s.dpr[i] / pb - s.bp[i];"),
    ("ab2_is_euler", "test_oracle_pins.py",
     "*rho = r + dxi * (1.5 * fr - 0.5 * *frp);", "*rho = r + dxi * fr;"),
    ("sort_unstable_on_ties", "test_oracle_pins.py",
     "dst[k++] = (key[src[j]] < key[src[i]]) ? src[j++] : src[i++];",
     "dst[k++] = (key[src[j]] <= key[src[i]]) ? src[j++] : src[i++];"),
    ("binning_without_half", "test_oracle_pins.py",
     "return (int64_t)floor(xi / dxi + 0.5);", "return (int64_t)floor(xi / dxi);"),
    ("ion_psi_outside_constant", "test_oracle_pins.py", "    return -q * log(rho);", "    return -q * log(rho_max);"),
    # the B^(p) solves (Eq. ai_bi: banded elimination, App. A shooting)
    ("band_source_a_factor", "test_oracle_pins.py",
     "x[ra] = 0.25 * (2.0 * Bi + Ai * Ci);", "x[ra] = 0.25 * (2.0 * Bi - Ai * Ci);"),
    ("band_matrix_m21_sign", "test_oracle_pins.py",
     "SET(rb, ca0, 0.5 * Ai * r * r * r);", "SET(rb, ca0, -0.5 * Ai * r * r * r);"),
    ("band_outer_condition_on_b", "test_oracle_pins.py",
     "SET(m - 1, m - 2, 1.0);  /* a_N = 0 */", "SET(m - 1, m - 1, 1.0);"),
    ("band_no_pivoting", "test_oracle_pins.py",
     "            if (fabs(AB(r, k)) > best) {", "            if (0) {"),
    ("shooting_m12", "test_oracle_pins.py", "double m12 = 0.5 * Ai / r;", "double m12 = 0.5 * Ai * r;"),
    ("shooting_start_K", "test_oracle_pins.py",
     "K[0] = 1.0; U[0] = 0.0; T[0] = 0.0; P[0] = 0.0;", "K[0] = 1.0; U[0] = 1.0; T[0] = 0.0; P[0] = 0.0;"),
    ("guard_disabled", "test_oracle_pins.py",
     "static int ring_fields_ok(const slice_ws *s)\n{", "static int ring_fields_ok(const slice_ws *s)\n{\n    return 1;"),
    # fields at an arbitrary radius (a9)
    ("fields_at_psi_without_ions", "test_oracle_pins.py",
     "*psi = (s->Ltot - s->L[k]) + S * log(x) + ion_psi(x, dens, rho_max);", "*psi = (s->Ltot - s->L[k]) + S * log(x);"),
    ("fields_at_dzeta_index", "test_oracle_pins.py",
     "    *dpr = (S - ion_enclosed(x, dens, rho_max)) / x;\n    *dpz = -(s->Ttot - s->T[k]);",
     "    *dpr = (S - ion_enclosed(x, dens, rho_max)) / x;\n    *dpz = -(s->Ttot - s->T[k > 0 ? k - 1 : 0]);"),
    ("axis_dzeta_zero", "test_oracle_pins.py", "*dpz = -(s->Ttot - s->T[0]);", "*dpz = 0.0;"),
    ("axis_psi_without_rings", "test_oracle_pins.py",
     "*psi = s->Ltot + ion_psi(0.0, dens, rho_max);", "*psi = ion_psi(0.0, dens, rho_max);"),
    ("fields_at_bp_region", "test_oracle_pins.py",
     "*bp = s->a[k] * x + s->b[k] / x;", "*bp = s->a[k > 0 ? k - 1 : 0] * x + s->b[k > 0 ? k - 1 : 0] / x;"),
    # the two-species march (orc_run_ions)
    ("ions_axis_value_psi", "test_oracle_ions.py",
     "me->psi[i] = me->psi_o[i] + sp_interp(ot, ot->psi_o, ot->Ltot, 0, 0.0, x);",
     "me->psi[i] = me->psi_o[i] + sp_interp(ot, ot->psi_o, 0.0, 0, 0.0, x);"),
    ("ions_no_edge_node", "test_oracle_ions.py", "if (x >= s->edge || !(s->edge > rl))", "if (1)"),
    ("ions_interp_weight_swapped", "test_oracle_ions.py",
     "return Fl + (Fh - Fl) * (x - rl) / (rh - rl);", "return Fl + (Fh - Fl) * (rh - x) / (rh - rl);"),
    ("ions_half_weight", "test_oracle_ions.py", "cw[n + j] = -w0[j];", "cw[n + j] = -0.5 * w0[j];"),
    ("ions_no_self_weight", "test_oracle_ions.py", "ch[n + j] = -w0[n + j];", "ch[n + j] = 0.0;"),
    ("ions_psibar_without_qm", "test_oracle_ions.py",
     "double pb = 1.0 - me->qm * me->psi[i];", "double pb = 1.0 + me->psi[i];"),
    ("ions_push_without_qm", "test_oracle_ions.py",
     "double fu = -me->qm * (me->gam[i] * me->dpr[i] / pb - (me->bp[i] + me->bb[i]));",
     "double fu = (me->gam[i] * me->dpr[i] / pb - (me->bp[i] + me->bb[i]));"),
    ("ions_without_bp", "test_oracle_ions.py",
     "io->bp[i] = sp_interp(e, e->bp, 0.0, 3, bk[n], io->r[i]);", "io->bp[i] = 0.0;"),
    ("ions_no_bp_beyond_electrons", "test_oracle_ions.py", "return bN / x;", "return 0.0;"),
    ("beam_sees_electrons_only", "test_oracle_ions.py",
     "            for (int s = 0; s < 2; ++s) {\n                double a1, a2, a3;",
     "            for (int s = 0; s < 1; ++s) {\n                double a1, a2, a3;"),
    ("beam_without_bp_with_ions", "test_oracle_ions.py",
     "bpv = ak[k] * x + bk[k] / x;", "bpv = 0.0;"),
    ("ions_dzeta_axis_value", "test_oracle_ions.py",
     "me->dpz[i] = me->dpz_o[i] + sp_interp(ot, ot->dpz_o, -ot->Ttot, 2, 0.0, me->r[i]);",
     "me->dpz[i] = me->dpz_o[i] + sp_interp(ot, ot->dpz_o, 0.0, 2, 0.0, me->r[i]);"),
    ("ions_outside_dpr_zero", "test_oracle_ions.py",
     "if (which == 1) return s->Stot / x;", "if (which == 1) return 0.0;"),
    ("ions_own_dpr_without_self", "test_oracle_ions.py",
     "s->dpr_o[i] = (s->S[i] + s->ch[i]) / r;", "s->dpr_o[i] = s->S[i] / r;"),
    ("ions_own_dzeta_without_self", "test_oracle_ions.py",
     "s->dpz_o[i] = -(above + (1.0 - s->ch[i] / s->c[i]) * s->t[i]);", "s->dpz_o[i] = -(above + s->t[i]);"),
    ("profile_ignored", "test_oracle_ions.py",
     "double dens_j = p->cell_density ? p->cell_density[j] : p->density;", "double dens_j = p->density;"),
    # RK4 (orc_run, integrator rk4)
    ("rk4_half_step_source_slice_n", "test_oracle_rk4.py",
     "rc = slice_core(&s, ord_s, rs, us, w, wh, dens, rho_max, &bs, &bsn, 0.5, 0.5, NULL, dxi);",
     "rc = slice_core(&s, ord_s, rs, us, w, wh, dens, rho_max, &bs, NULL, 1.0, 0.0, NULL, dxi);"),
    ("rk4_last_stage_source_slice_n", "test_oracle_rk4.py",
     "rc = slice_core(&s, ord_s, rs, us, w, wh, dens, rho_max, &bsn, NULL, 1.0, 0.0, NULL, dxi);",
     "rc = slice_core(&s, ord_s, rs, us, w, wh, dens, rho_max, &bs, NULL, 1.0, 0.0, NULL, dxi);"),
    ("rk4_equal_stage_weights", "test_oracle_rk4.py", "ws[3] = {2.0, 2.0, 1.0}", "ws[3] = {1.0, 1.0, 1.0}"),
    ("rk4_stage_steps", "test_oracle_rk4.py", "cs[3] = {0.5, 0.5, 1.0}", "cs[3] = {0.5, 1.0, 1.0}"),
    ("rk4_first_stage_weight", "test_oracle_rk4.py", "sum_r[id] = ksr[id];", "sum_r[id] = 2.0 * ksr[id];"),
    # the axis: a stage state below it evaluated mirrored, the derivative
    # mirrored back (r and u parts), and the reflected AB2 history
    ("rk4_stage_rho_derivative_not_mirrored_back", "test_oracle_rk4.py",
     "ksr[id] = sg[id] * (s.u[i] / pb);", "ksr[id] = (s.u[i] / pb);"),
    ("rk4_stage_u_derivative_not_mirrored_back", "test_oracle_rk4.py",
     "ksu[id] = sg[id] * (s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]));",
     "ksu[id] = (s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]));"),
    ("ab2_axis_history_not_flipped", "test_oracle_pins.py",
     "        *frp = -*frp;\n        *fup = -*fup;\n", ""),
    ("ab2_axis_u_history_not_flipped", "test_oracle_pins.py", "        *fup = -*fup;\n", ""),
    ("ab2_axis_u_not_reflected", "test_oracle_pins.py", "        *ur = -*ur;\n", ""),
    # beam grids (Sec. IV)
    ("grid_extent_without_margin", "test_oracle_grid.py",
     "agR[b] = (agR[b] > 1e-12 ? agR[b] : 1e-12) * (1.0 + 1.0 / nr);",
     "agR[b] = (agR[b] > 1e-12 ? agR[b] : 1e-12) * (1.0 + 1e-9);"),
    ("grid_deposit_on_the_node_below", "test_oracle_grid.py",
     "int32_t j = ag_cell(bs.r[q], dr, nr) + 1;", "int32_t j = ag_cell(bs.r[q], dr, nr);"),
    ("grid_node_field_without_2pi", "test_oracle_grid.py",
     "B[j] = acc / (ORC_2PI * dxi * ((double)j * dr));", "B[j] = acc / (dxi * ((double)j * dr));"),
    ("grid_no_field_beyond", "test_oracle_grid.py", "return B[g->nr] * R / rho;", "return 0.0;"),
    ("grid_ring_field_left_node", "test_oracle_grid.py",
     "return (1.0 - t) * B[j] + t * B[j + 1];", "return B[j];"),
    ("grid_gather_left_node", "test_oracle_grid.py",
     "psi = (1.0 - t) * F0[0] + t * F1[0];\n                dpr = (1.0 - t) * F0[1] + t * F1[1];\n"
     "                dpz = (1.0 - t) * F0[2] + t * F1[2];",
     "psi = F0[0];\n                dpr = F0[1];\n                dpz = F0[2];"),
    ("grid_nodes_without_beam_field", "test_oracle_grid.py",
     "F[3] = bpv + (j > 0 ? ag_field(&ag, x) : 0.0);", "F[3] = bpv;"),
    ("grid_all_species_on_one_grid", "test_oracle_grid.py",
     "int32_t b = p->beam_species ? p->beam_species[bs.idx[q]] : 0;\n                double dr = agR[b] / nr;",
     "int32_t b = 0;\n                double dr = agR[b] / nr;"),
    ("regular_grid_ignored", "test_oracle_grid.py", "                    agR[b] = p->grid_rmax;\n", ""),
    ("regular_grid_unchecked", "test_oracle_grid.py",
     "                    if (!(agR[b] < p->grid_rmax))\n                        rc = ORC_EINVAL;\n", ""),
    ("grid_one_extent_for_all", "test_oracle_grid.py",
     "if (p->beam_r[k] > agR[b]) agR[b] = p->beam_r[k];",
     "for (int32_t b2 = 0; b2 < p->n_species; ++b2) if (p->beam_r[k] > agR[b2]) agR[b2] = p->beam_r[k];"),
]

# the Boris push (oracle/beam_push.py): (name, original text, planted text)
PY_CASES = [
    ("second_half_kick_missing", "    return upl + h * E", "    return upl"),
    ("rotation_gamma_before_the_kick", "    gm = np.sqrt(1.0 + np.sum(um * um, axis=0))",
     "    gm = np.sqrt(1.0 + np.sum(u * u, axis=0))"),
    ("rotation_s_not_normalised", "    s = 2.0 * t / (1.0 + np.sum(t * t, axis=0))", "    s = t"),
    ("rotation_cross_order", "    up = um + np.cross(um, t, axis=0)", "    up = um + np.cross(t, um, axis=0)"),
    ("er_without_btheta", "    er = wr + bt", "    er = wr"),
    ("er_minus_btheta", "    er = wr + bt", "    er = wr - bt"),
    ("b_sign", "    B = np.stack([-bt * s, bt * c, np.zeros_like(bt)])",
     "    B = np.stack([bt * s, -bt * c, np.zeros_like(bt)])"),
    ("ez_sign", "    E = np.stack([er * c, er * s, ez])", "    E = np.stack([er * c, er * s, -ez])"),
    ("xi_drift_sign", '"xi": state["xi"] + dt * (1.0 - un[2] / g)', '"xi": state["xi"] - dt * (1.0 - un[2] / g)'),
    ("position_with_old_gamma", "    g = np.sqrt(1.0 + np.sum(un * un, axis=0))\n    out",
     "    g = np.sqrt(1.0 + np.sum(u * u, axis=0))\n    out"),
    ("kick_of_a_full_step", "    h = 0.5 * np.asarray(q, dtype=np.float64) * dt",
     "    h = np.asarray(q, dtype=np.float64) * dt"),
    ("x_moves_with_uy", '"x": state["x"] + dt * un[0] / g', '"x": state["x"] + dt * un[1] / g'),
]


def _run_c_case(case, workdir):
    name, pin_file, old, new = case
    from oracle import oracle as orc
    src = open(os.path.join(ORACLE, "wake_oracle.c")).read()
    assert src.count(old) == 1, f"{name}: the original text must occur once"
    d = os.path.join(workdir, name)
    os.makedirs(d)
    shutil.copy(os.path.join(ORACLE, "wake_oracle.h"), d)
    with open(os.path.join(d, "wake_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(d, "liboracle.so")
    subprocess.check_call(["gcc", *orc.GCC_FLAGS, "-o", lib, os.path.join(d, "wake_oracle.c"), "-lm"])
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join("tests", pin_file), "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    failed = [ln.split("::", 1)[1].split(" ")[0] for ln in r.stdout.splitlines() if ln.startswith("FAILED")]
    return r.returncode, failed, r.stdout[-400:]


@pytest.fixture(scope="module")
def c_results(tmp_path_factory):
    work = str(tmp_path_factory.mktemp("planted"))
    workers = max(1, min(len(C_CASES), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        futs = {c[0]: ex.submit(_run_c_case, c, work) for c in C_CASES}
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name", [c[0] for c in C_CASES])
def test_a_planted_mistake_in_the_c_oracle_fails_a_pin(c_results, name):
    rc, failed, tail = c_results[name]
    assert rc == 1 and failed, (name, rc, tail)


def _pin_module():
    spec = importlib.util.spec_from_file_location("_push_pins", os.path.join(ROOT, "tests", "test_oracle_beam_push.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", PY_CASES, ids=[c[0] for c in PY_CASES])
def test_a_planted_mistake_in_the_push_oracle_fails_a_pin(name, old, new):
    src = open(os.path.join(ORACLE, "beam_push.py")).read()
    assert src.count(old) == 1
    planted = types.ModuleType("_planted_beam_push")
    exec(compile(src.replace(old, new), "planted_beam_push.py", "exec"), planted.__dict__)
    pins = _pin_module()
    pins.bp = planted
    failed = []
    for t in [getattr(pins, k) for k in dir(pins) if k.startswith("test_")]:
        try:
            t()
        except AssertionError:
            failed.append(t.__name__)
    assert failed, name
