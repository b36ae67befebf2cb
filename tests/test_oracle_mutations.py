"""The oracle's pins must catch plausible mistakes: each case plants one
slip in a temporary copy of the oracle (CPU only) and checks that the pin
suite fails on it."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "weight_factor_2": ("w = 2.0 * sinc_step * np.cosh(u)", "w = 1.0 * sinc_step * np.cosh(u)"),
    "full_weight_at_q0": ("w[0] = sinc_step / (t_scale", "w[0] = 2.0 * sinc_step / (t_scale"),
    "window_off_by_one": ("return gq[N - m: 2 * N - m].copy()", "return gq[N - m + 1: 2 * N - m + 1].copy()"),
    "vertex_not_centre_grid": ("xt = (np.arange(2 * N, dtype=np.float64) - N + 0.5) * h",
                               "xt = (np.arange(2 * N, dtype=np.float64) - N) * h"),
    "no_multiplicity_weight": ("Aw = (ncols[a] * np.sqrt(count)[:, None]).T", "Aw = ncols[a].T"),
    "core_mode_swap": ("p1 = P[0][:, tcol[sl, 0]] * xi[sl]", "p1 = P[0][:, tcol[sl, 1]] * xi[sl]"),
    "rank_rule_squared": ("if math.sqrt(tail[r]) <= eps * math.sqrt(total):", "if tail[r] <= eps * total:"),
    "defect_sign": ("return defect.charge - blocks[defect.block].charge",
                    "return blocks[defect.block].charge - defect.charge"),
    "norms_not_in_xi": ("xin = xin * norms[a][tcol[:, a]]", "xin = xin"),
    "yukawa_printed_exponent": ("w = w * np.exp(-(kappa * kappa) / (4.0 * t * t))",
                                "w = w * np.exp(-(kappa * kappa) / (t * t))"),
    "yukawa_factor_inverted": ("w = w * np.exp(-(kappa * kappa) / (4.0 * t * t))",
                               "w = w * np.exp(-(kappa * kappa) * (t * t) / 4.0)"),
    "yukawa_unscreened_kernel": ("        return 1.0 / (r * r * r)\n    return np.exp(-kappa * r) / r",
                                 "        return 1.0 / (r * r * r)\n    return 1.0 / r"),
    "galerkin_cell_shift": ("g[q, j] = c * gaussian_cell_average(float(t[q]), (j - N) * h, (j - N + 1) * h)",
                            "g[q, j] = c * gaussian_cell_average(float(t[q]), (j - N + 0.5) * h, (j - N + 1.5) * h)"),
    "als_unweighted_terms": ("al = ncols[l][tcol[sl, l]].T * xin[sl]", "al = ncols[l][tcol[sl, l]].T"),
    "slater_prefactor": ("a = (kappa / math.sqrt(math.pi)) / (t * t)", "a = (2.0 * kappa / math.sqrt(math.pi)) / (t * t)"),
    "dipole_power": ("a = (4.0 / math.sqrt(math.pi)) * t * t", "a = (4.0 / math.sqrt(math.pi)) * t"),
    "tucker_bhat_unscaled": ("Bhat2 += float(np.sum(core * core)) * (sc[0] * sc[1] * sc[2]) ** 2",
                             "Bhat2 += float(np.sum(core * core))"),
    "tucker_defect_new_charge": ("terms.append(([side(ms[a]) for a in range(3)], defect_charge(d, blocks) * b,",
                                 "terms.append(([side(ms[a]) for a in range(3)], d.charge * b,"),
    "tucker_core_mode_swap": ("P = [out[\"Z\"][a].T @ F[a] for a in range(3)]",
                              "P = [out[\"Z\"][a].T @ F[(a + 1) % 3] for a in range(3)]"),
    "galerkin_no_hadamard": ('M = [np.einsum("ki,mi,ia->kma", basis[l], basis[l], Z[l], optimize=True) for l in range(3)]',
                             'M = [np.einsum("ki,mi,ia->kma", basis[l], np.ones_like(basis[l]), Z[l], optimize=True) '
                             'for l in range(3)]'),
    "galerkin_mode_swap": ('M = [np.einsum("ki,mi,ia->kma", basis[l], basis[l], Z[l], optimize=True) for l in range(3)]',
                           'M = [np.einsum("ki,mi,ia->kma", basis[l], basis[l], Z[(l + 1) % 3], optimize=True) '
                           'for l in range(3)]'),
    "tucker_reference_unprojected": ("h = Z.T @ g.T                               # (r, R): Z^T g_q",
                                     "h = Z.T @ (g / np.sqrt((g * g).sum(1))[:, None]).T"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pin_suite_catches_planted_mistake(tmp_path, name):
    old, new = MUTATIONS[name]
    for d in ("oracle", "tests", "paper_1411_1994_gb300"):
        os.makedirs(tmp_path / d, exist_ok=True)
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), tmp_path / "oracle")
    src = open(os.path.join(ROOT, "oracle", "lattice_oracle.py")).read()
    assert old in src
    (tmp_path / "oracle" / "lattice_oracle.py").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "paper_1411_1994_gb300", "workloads.py"), tmp_path / "paper_1411_1994_gb300")
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        str(tmp_path / "tests" / "test_oracle_pins.py")],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation {name} survived the pins:\n{r.stdout[-2000:]}"
