"""The oracle's pins reject an oracle with a planted mistake.

Each case copies oracle/gs_oracle.cpp, plants one plausible mistake in the
copy (a dropped term, a flipped sign, a transposed operand, a wrong index or
factor), builds it, and runs the pins of that part of the oracle (elements,
contact, integration and adjoint: tests/test_oracle_pins.py; air, rigid bodies,
actuation sequences: their own pin files) against that build (GS_ORACLE_LIB):
at least one pin must fail.  An unchanged copy built the same way must pass all
four pin files, so a failure is the planted mistake's doing.  The committed
oracle source is never modified.  CPU only."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gs_oracle.cpp")
HDR = os.path.join(ROOT, "oracle", "gs_oracle.h")

# name: (text in the oracle, its replacement, occurrences replaced)
MUTANTS = {
    # App. A.1 stable neo-Hookean P: the mu F / (I_C + 1) term dropped from the tet force
    "tet_P_term_dropped": ("const T a = mu * (1.0 - 1.0 / (Ic + 1.0));\n    const T b = lam * (J - alpha);\n    T P[3][3];",
                           "const T a = mu;\n    const T b = lam * (J - alpha);\n    T P[3][3];", 1),
    # H = -V P Dm^-T with Dm^-1 in place of its transpose
    "tet_Dm_untransposed": ("P[r][0] * Dminv[3 * c] + P[r][1] * Dminv[3 * c + 1] + P[r][2] * Dminv[3 * c + 2]",
                            "P[r][0] * Dminv[c] + P[r][1] * Dminv[3 + c] + P[r][2] * Dminv[6 + c]", 1),
    # the rest-stable alpha = 1 + 3 mu / (4 lambda) with a wrong factor (energy and force alike)
    "tet_alpha_factor": ("0.75 * mu / lam", "0.5 * mu / lam", 2),
    # membrane dJ/df_0 = f_1 x n with the cross product's operands swapped (a sign)
    "tri_dJ_sign": ("vcross(f1, n, dJ0);", "vcross(n, f1, dJ0);", 1),
    # lumped mass: a quarter of each tet's mass per corner, here a third
    "mass_lumping_factor": ("mass[m->tets[4 * e + c]] += tet_rho[e] * (r.tet_V[e] / 4.0);",
                            "mass[m->tets[4 * e + c]] += tet_rho[e] * (r.tet_V[e] / 3.0);", 1),
    # contact damping k_d dC/dt with dC/dt = -v.n: the sign flipped
    "contact_damping_sign": ("const T fn = ke * C - kd * vn;", "const T fn = ke * C + kd * vn;", 1),
    # stick friction -k_f v_s: the sign flipped
    "friction_stick_sign": ("for (int k = 0; k < 3; ++k) f[k] -= kf * vs[k];",
                            "for (int k = 0; k < 3; ++k) f[k] += kf * vs[k];", 1),
    # Bridson bending sin(phi / 2 + alpha): the half angle lost
    "bending_half_angle": ("fsin(0.5 * phi + act)", "fsin(phi + act)", 1),
    # bending direction u_3 with a wrong edge end (index)
    "bending_u3_index": ("f[6 + k] = s * (p14 * g1[k] + p24 * g2[k]);",
                         "f[6 + k] = s * (p13 * g1[k] + p24 * g2[k]);", 1),
    # semi-implicit Euler (App. B): x+ from the old velocity (explicit Euler)
    "euler_old_velocity": (
        "            v[3 * (size_t)i + k] = v[3 * (size_t)i + k] + dt * (w[i] * f[3 * (size_t)i + k] + (dyn ? m->gravity[k] : 0.0));\n"
        "            x[3 * (size_t)i + k] = x[3 * (size_t)i + k] + dt * v[3 * (size_t)i + k];",
        "            x[3 * (size_t)i + k] = x[3 * (size_t)i + k] + dt * v[3 * (size_t)i + k];\n"
        "            v[3 * (size_t)i + k] = v[3 * (size_t)i + k] + dt * (w[i] * f[3 * (size_t)i + k] + (dyn ? m->gravity[k] : 0.0));",
        1),
    # gravity applied to kinematic (pinned) nodes too
    "gravity_on_pinned": ("(dyn ? m->gravity[k] : 0.0)", "m->gravity[k]", 1),
    # discrete adjoint (App. B): c_u = -dl/du+ - dt dl/dq+ without its dt term
    "adjoint_dt_term_dropped": ("cu[i] = -lu[i] - dt * lq[i];", "cu[i] = -lu[i];", 1),
    # the sphere's contact normal pointing inwards
    "sphere_normal_sign": ("T nn[3] = {d[0] / dist, d[1] / dist, d[2] / dist};",
                           "T nn[3] = {-d[0] / dist, -d[1] / dist, -d[2] / dist};", 1),
    # Coulomb slip friction mu |f_n| v_s / |v_s| without the normalisation
    "slip_not_normalised": ("const T scale = muf * afn / vsl;", "const T scale = muf * afn;", 1),
    # hinge actuation inside the half angle: sin((phi + a) / 2) for sin(phi / 2 + a)
    "hinge_act_halved": ("fsin(0.5 * phi + act)", "fsin(0.5 * (phi + act))", 1),
    # the membrane's rest-stable alpha = 1 + 2 mu / (3 lambda) with the tet's factor
    "tri_alpha_factor": ("(2.0 / 3.0) * mu / lam", "0.75 * mu / lam", 2),
    # cloth mass lumping: a third of each triangle's mass per corner, here a quarter
    "cloth_mass_lumping": ("mass[m->tris[3 * t + c]] += tri_rho[t] * (r.tri_A[t] / 3.0);",
                           "mass[m->tris[3 * t + c]] += tri_rho[t] * (r.tri_A[t] / 4.0);", 1),
    # density gradient rho_bar_e = (V_e / 4) sum m_bar_i with a wrong share
    "density_grad_factor": ("g->tet_rho[e] = s * (r.tet_V[e] / 4.0);", "g->tet_rho[e] = s * (r.tet_V[e] / 3.0);", 1),
    # dL/dw_i += -dt c_u,i . f_i with its sign flipped
    "adjoint_w_term_sign": ("w_b[i] += -dt * cu[3 * i + k] * f_n[3 * i + k];",
                            "w_b[i] += dt * cu[3 * i + k] * f_n[3 * i + k];", 1),
    # m_bar = -w^2 w_bar (d(1/m)/dm) with its sign flipped
    "mass_grad_sign": ("m_b[i] = -w[i] * w[i] * w_b[i];", "m_b[i] = w[i] * w[i] * w_b[i];", 1),
    # the loss seed dL/dx(S) = 2 (x - x*) without its factor 2
    "loss_seed_factor": ("lq[i] = 2.0 * d;", "lq[i] = d;", 1),
    # rest volume det(Dm) / 6 with a wrong factor
    "tet_volume_factor": ("*V = det / 6.0;", "*V = det / 2.0;", 1),
    # node gather: a tet's corner forces added to the next corner's node
    "tet_gather_corner": ("f[3 * (size_t)m->tets[4 * e + c] + k] += fe[12 * (size_t)e + 3 * c + k];",
                          "f[3 * (size_t)m->tets[4 * e + (c + 1) % 4] + k] += fe[12 * (size_t)e + 3 * c + k];", 1),
    # node gather: a hinge's corner forces added to the next corner's node
    "hinge_gather_corner": ("f[3 * (size_t)m->hinges[4 * h + c] + k] += fe[12 * (size_t)h + 3 * c + k];",
                            "f[3 * (size_t)m->hinges[4 * h + (c + 1) % 4] + k] += fe[12 * (size_t)h + 3 * c + k];", 1),
    # adjoint: a tet's corner x_bar added to the next corner's node
    "adjoint_tet_scatter_corner": (
        "lq_new[3 * (size_t)m->tets[4 * e + c] + k] += xb_e[12 * (size_t)e + 3 * c + k];",
        "lq_new[3 * (size_t)m->tets[4 * e + (c + 1) % 4] + k] += xb_e[12 * (size_t)e + 3 * c + k];", 1),
    # sphere penetration r - |x - c| with its sign flipped
    "sphere_depth_sign": ("const T C = m->sphere_r - dist;", "const T C = dist - m->sphere_r;", 1),
    # the stick / slip test reversed
    "stick_slip_threshold": ("if (val(kf) * vsl_val <= val(muf) * val(afn)) {",
                             "if (val(kf) * vsl_val >= val(muf) * val(afn)) {", 1),
    # membrane corner forces with half the rest area
    "tri_force_area": ("const T h = -A * (P[r][0] * Dminv[2 * cc] + P[r][1] * Dminv[2 * cc + 1]);",
                       "const T h = -0.5 * A * (P[r][0] * Dminv[2 * cc] + P[r][1] * Dminv[2 * cc + 1]);", 1),
    # Bridson direction u_4 with one term's sign flipped
    "bending_u4_sign": ("f[9 + k] = s * (-(p13 * g1[k]) - p23 * g2[k]);",
                        "f[9 + k] = s * ((p13 * g1[k]) - p23 * g2[k]);", 1),
    # density gradient summing one corner's m_bar four times
    "density_grad_corner": ("s += m_b[m->tets[4 * e + c]];", "s += m_b[m->tets[4 * e]];", 1),
    # adjoint force seed f_bar = -dt W c_u without the inverse mass
    "adjoint_seed_no_mass": ("y[3 * i + k] = -dt * w[i] * cu[3 * i + k];", "y[3 * i + k] = -dt * cu[3 * i + k];", 1),
    # adjoint: a triangle's corner x_bar added to the next corner's node
    "adjoint_tri_scatter_corner": (
        "lq_new[3 * (size_t)m->tris[3 * e + c] + k] += xb_e[9 * (size_t)e + 3 * c + k];",
        "lq_new[3 * (size_t)m->tris[3 * e + (c + 1) % 3] + k] += xb_e[9 * (size_t)e + 3 * c + k];", 1),
    # adjoint: a hinge's corner x_bar added to the next corner's node
    "adjoint_hinge_scatter_corner": (
        "lq_new[3 * (size_t)m->hinges[4 * h + c] + k] += xb_e[12 * (size_t)h + 3 * c + k];",
        "lq_new[3 * (size_t)m->hinges[4 * h + (c + 1) % 4] + k] += xb_e[12 * (size_t)h + 3 * c + k];", 1),
    # dL/dmu and dL/dlambda of a tet swapped
    "adjoint_mu_lambda_swapped": ("tmu_b[e] += pb[0]; tlam_b[e] += pb[1];", "tmu_b[e] += pb[1]; tlam_b[e] += pb[0];", 1),
    # the contact force's dependence on v dropped from the velocity adjoint
    "adjoint_contact_v_dropped": ("lq_new[3 * i + k] += xb[k]; lu_new[3 * i + k] += xb[3 + k];",
                                  "lq_new[3 * i + k] += xb[k];", 1),
    # the bending stiffness gradient dropped
    "adjoint_kb_dropped": ("kb_b[h] += pb[0]; hact_b[h] += pb[1];", "hact_b[h] += pb[1];", 1),
    # dl/du- = -c_u replaced by -c_q (the wrong multiplier)
    "adjoint_velocity_multiplier": ("{ lq_new[i] = -cq[i]; lu_new[i] = -cu[i]; }",
                                    "{ lq_new[i] = -cq[i]; lu_new[i] = -cq[i]; }", 1),
}
# the same for the air model, the rigid-body step and the actuation sequence,
# each against its own pins: name: (text, replacement, occurrences, pin file)
MUTANTS_MORE = {
    # flat-plate lift with its direction reversed
    "air_lift_sign": ("F[k] = F[k] - c * (q * N[k] - s * vr[k]);", "F[k] = F[k] + c * (q * N[k] - s * vr[k]);", 1,
                      "test_oracle_air.py"),
    # the plate's velocity through the air: the wind added instead of subtracted
    "air_wind_sign": ("vr[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0 - wind[k];",
                      "vr[k] = (v[k] + v[3 + k] + v[6 + k]) / 3.0 + wind[k];", 1, "test_oracle_air.py"),
    # a triangle's air force shared over its corners by halves instead of thirds
    "air_corner_share": ("for (int k = 0; k < 3; ++k) f[3 * c + k] = F[k] / 3.0;",
                         "for (int k = 0; k < 3; ++k) f[3 * c + k] = F[k] / 2.0;", 1, "test_oracle_air.py"),
    # quaternion update r + dt/2 (0, omega) r with dt in place of dt/2
    "rigid_quat_half_step": ("0.5 * dt *", "1.0 * dt *", 2, "test_oracle_rigid.py"),
    # Newton-Euler: tau - omega x (I omega) with the gyroscopic term's sign flipped
    "rigid_gyroscopic_sign": ("h[i] = tau[i] - wL[i];", "h[i] = tau[i] + wL[i];", 1, "test_oracle_rigid.py"),
    # world inertia R I_b R^T taken as R^T I_b R
    "rigid_inertia_transposed": ("acc += R[i][a] * Ib[a][c] * R[j][c];", "acc += R[a][i] * Ib[a][c] * R[c][j];", 1,
                                 "test_oracle_rigid.py"),
    # a contact point's moment d x f with the operands swapped (a sign)
    "rigid_moment_sign": ("vcross(d, fc, td);", "vcross(fc, d, td);", 1, "test_oracle_rigid.py"),
    # Newton: the contact force multiplied by the mass instead of divided
    "rigid_force_times_mass": ("vo[i] = v[i] + dt * (sc->gravity[i] + F[i] / m);",
                               "vo[i] = v[i] + dt * (sc->gravity[i] + F[i] * m);", 1, "test_oracle_rigid.py"),
    # flat-plate lift without the area normalisation of N
    "air_lift_area": ("const T c = k_lift * s / (fsqrt(A2) * fsqrt(q));", "const T c = k_lift * s / fsqrt(q);", 1,
                      "test_oracle_air.py"),
    # the air force's dependence on the corner velocities dropped from the adjoint
    "adjoint_air_v_dropped": ("lu_new[3 * (size_t)m->tris[3 * e + c] + k] += xb_e[18 * (size_t)e + 9 + 3 * c + k];",
                              "lu_new[3 * (size_t)m->tris[3 * e + c] + k] += 0.0;", 1, "test_oracle_air.py"),
    # the row of the actuation sequence added at half weight
    "act_seq_scale": ("ta[e] += tseq[(size_t)n * m->n_tets + e];", "ta[e] += 0.5 * tseq[(size_t)n * m->n_tets + e];",
                      1, "test_oracle_actuation.py"),
}
PIN_FILES = ("test_oracle_pins.py", "test_oracle_air.py", "test_oracle_rigid.py", "test_oracle_actuation.py")


def _build(tmp_path, name, text=None, repl=None, count=0):
    src = open(SRC).read()
    if text is not None:
        assert src.count(text) == count, (name, src.count(text))
        src = src.replace(text, repl)
    d = tmp_path / name
    d.mkdir()
    (d / "gs_oracle.cpp").write_text(src)
    (d / "gs_oracle.h").write_text(open(HDR).read())
    so = d / "liboracle.so"
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so),
                           str(d / "gs_oracle.cpp")])
    return str(so)


def _pins(lib_path, files=("test_oracle_pins.py",)):
    env = dict(os.environ, GS_ORACLE_LIB=lib_path, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", *[os.path.join(ROOT, "tests", f) for f in files], "-x", "-q",
           "-p", "no:cacheprovider"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)




# the renderer's oracle (plain PyTorch) against tests/test_oracle_render.py: a
# mutated copy of oracle/render_oracle.py is registered as oracle.render_oracle
# before the pins import it
RENDER_SRC = os.path.join(ROOT, "oracle", "render_oracle.py")
RENDER_MUTANTS = {
    # coverage sigmoid(+-d^2 / sigma): inside and outside swapped
    "render_coverage_sign": ("tv = torch.where(inside, d2, -d2) / spec.sigma",
                             "tv = torch.where(inside, -d2, d2) / spec.sigma"),
    # silhouette as the probabilistic union 1 - prod(1 - D): a clamped sum instead
    "render_union_as_sum": ("A = 1.0 - torch.prod(q, dim=1)", "A = D.sum(dim=1).clamp(max=1.0)"),
    # perspective-correct depth 1/z = sum w_k / z_k: z interpolated affinely instead
    "render_affine_depth": ("iz = (wc / zs[None]).sum(-1)", "iz = 1.0 / (wc * zs[None]).sum(-1)"),
    # barycentric weights with two corners' weights swapped (an index)
    "render_barycentric_order": ("w = torch.stack([_cross2(pb, pc), _cross2(pc, pa), _cross2(pa, pb)], dim=-1)",
                                 "w = torch.stack([_cross2(pc, pa), _cross2(pb, pc), _cross2(pa, pb)], dim=-1)"),
    # world to camera with the rotation transposed
    "render_rotation_transposed": ("xc = x @ R.T + t", "xc = x @ R + t"),
    # normalised depth with nearer = smaller, so the farthest covering triangle wins
    "render_depth_order": ("zh = (cam.z_far - zp) / (cam.z_far - cam.z_near)",
                           "zh = (zp - cam.z_near) / (cam.z_far - cam.z_near)"),
}

_RENDER_BOOT = """
import importlib.util, sys
root, path, test = sys.argv[1:4]
sys.path.insert(0, root)
import oracle
spec = importlib.util.spec_from_file_location("oracle.render_oracle", path)
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.render_oracle"] = mod
spec.loader.exec_module(mod)
oracle.render_oracle = mod
import pytest
sys.exit(pytest.main([test, "-x", "-q", "-p", "no:cacheprovider"]))
"""


def _render_pins(tmp_path, name, text=None, repl=None):
    src = open(RENDER_SRC).read()
    if text is not None:
        assert src.count(text) == 1, name
        src = src.replace(text, repl)
    path = tmp_path / f"{name}.py"
    path.write_text(src)
    cmd = [sys.executable, "-c", _RENDER_BOOT, ROOT, str(path), os.path.join(ROOT, "tests", "test_oracle_render.py")]
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every copy built and run against its pins, several at a time (each
    run is its own process, one thread each)."""
    base = tmp_path_factory.mktemp("mutants")
    rbase = tmp_path_factory.mktemp("render_mutants")
    jobs = {"unchanged": lambda: _pins(_build(base, "unchanged"), PIN_FILES),
            "render:unchanged": lambda: _render_pins(rbase, "unchanged")}
    for name, (text, repl, count) in MUTANTS.items():
        jobs[name] = lambda n=name, t=text, r=repl, c=count: _pins(_build(base, n, t, r, c))
    for name, (text, repl, count, pins) in MUTANTS_MORE.items():
        jobs[name] = lambda n=name, t=text, r=repl, c=count, f=pins: _pins(_build(base, n, t, r, c), (f,))
    for name, (text, repl) in RENDER_MUTANTS.items():
        jobs["render:" + name] = lambda n=name, t=text, r=repl: _render_pins(rbase, n, t, r)
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futures = {k: ex.submit(f) for k, f in jobs.items()}
        return {k: f.result() for k, f in futures.items()}


def _caught(r):
    return r.returncode == 1 and "failed" in r.stdout


def test_unchanged_copies_pass_the_pins(outcomes):
    for k in ("unchanged", "render:unchanged"):
        assert outcomes[k].returncode == 0, (k, outcomes[k].stdout[-3000:])


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(outcomes, name):
    assert _caught(outcomes[name]), (name, outcomes[name].returncode, outcomes[name].stdout[-3000:])


@pytest.mark.parametrize("name", sorted(MUTANTS_MORE))
def test_planted_mistake_fails_its_own_pins(outcomes, name):
    assert _caught(outcomes[name]), (name, outcomes[name].returncode, outcomes[name].stdout[-3000:])


@pytest.mark.parametrize("name", sorted(RENDER_MUTANTS))
def test_planted_render_mistake_fails_a_pin(outcomes, name):
    r = outcomes["render:" + name]
    assert _caught(r), (name, r.returncode, r.stdout[-3000:])
