"""CPU-side checks of the C-ABI library (no GPU needed).

* the in-tree libsphdvr.so loads and exports every function include/sphdvr.h declares;
* argument validation paths return the documented status codes;
* the library's own look-up-table builder (host code) agrees with the oracle's
  table and reproduces the paper's printed E_{K,D} values (Sec. 5.2 figure).
"""
import ctypes
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad, simpson

import oracle

S = pytest.importorskip("paper_2401_02896_b300.sphdvr", reason="libsphdvr.so not built")
HERE = os.path.dirname(os.path.abspath(__file__))


def test_library_exports_every_declared_function():
    names = S.header_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(S.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings():
    for s in range(9):
        assert S.status_string(s) and S.status_string(s) != "unknown status"
    assert S.status_string(99) == "unknown status"
    assert "sm_103a" in S.version()


def test_create_without_cuda_device_reports_edevice():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_create(0)
    assert e.value.status == S.EDEVICE


@pytest.mark.parametrize("args", [("m4", 0, 3, 64), ("m4", 5, 3, 64), ("m4", 4, 0, 64), ("m4", 4, 7, 64),
                                  ("m4", 4, 3, 1), (9, 4, 3, 64)])
def test_lut_build_rejects_bad_arguments(args):
    with pytest.raises((S.SphdvrError, KeyError)) as e:
        S.sphdvr_lut_build(*args)
    if isinstance(e.value, S.SphdvrError):
        assert e.value.status == S.EINVAL


def test_null_handles_are_rejected():
    lib = S._lib
    assert lib.sphdvr_destroy(None) == S.EINVAL
    assert lib.sphdvr_lut_free(None) == S.EINVAL
    assert lib.sphdvr_dataset_free(None) == S.EINVAL
    assert lib.sphdvr_create(0, None) == S.EINVAL
    info = (ctypes.c_int64 * 8)()
    assert lib.sphdvr_dataset_info(None, info) == S.EINVAL


@pytest.mark.parametrize("kernel,K,D", [("m4", 4, 3), ("wendland_c2", 4, 3), ("wendland_c4", 4, 4), ("m4", 2, 2),
                                        ("m4", 3, 3)])
def test_library_table_matches_oracle_table(kernel, K, D):
    n = 129
    th, pc, err = S.sphdvr_lut_build(kernel, K, D, n)
    L = oracle.lut_build(kernel, K, D, n)
    e_o = L["err"][:-1]
    e_p = err[:-1]
    nb = L["normB"][:-1]
    # never noticeably worse than the oracle's optimum, per entry
    assert np.all(e_p <= e_o * (1 + 5e-3) + 1e-13 * nb)
    # the error the library reports is the error of the approximation it returns
    for j in [3, 40, 77, 120]:
        e_chk, _ = oracle.fixed_knots(kernel, K, D, L["lam"][j], th[j])
        assert abs(e_chk - err[j]) <= 1e-7 * nb[j] + 1e-12 * e_chk
    # last entry: zero function
    assert np.all(th[-1] == 0) and np.all(pc[-1] == 0)


@pytest.mark.parametrize("key", ["2,1", "4,3", "3,2", "4,4"])
def test_library_table_reproduces_printed_errors(key):
    table = json.load(open(os.path.join(HERE, "golden", "paper_error_table.json")))
    K, D = map(int, key.split(","))
    th, pc, err = S.sphdvr_lut_build("m4", K, D, 257)
    kap = math.sqrt(4 * math.pi * quad(lambda r: (r * oracle.kernel_w("m4", r)) ** 2, 0, 2, points=[1.0],
                                       epsabs=1e-16)[0])
    lam = np.arange(257) * 2.0 / 256
    E = math.sqrt(2 * math.pi * simpson(lam * err ** 2, x=lam)) / kap
    assert abs(E / table["E"][key] - 1) < 1.5e-4


def test_library_table_poly6_exact():
    th, pc, err = S.sphdvr_lut_build("poly6", 1, 6, 33)
    lam = np.arange(33) / 32.0
    for j in range(32):
        nb = math.sqrt(oracle.ray_norm2("poly6", lam[j]))
        assert err[j] <= 1e-10 * nb
        assert abs(th[j][0] - math.sqrt(1 - lam[j] ** 2)) < 1e-5


@pytest.mark.parametrize("key", ["2,1", "4,3", "3,2", "4,4", "1,6", "2,5"])
def test_lut_error_measure_reproduces_printed_errors(key):
    """sphdvr_lut_error_measure on the library's own table gives the paper's printed E_{K,D} (Sec. 5.2 figure)."""
    table = json.load(open(os.path.join(HERE, "golden", "paper_error_table.json")))
    K, D = map(int, key.split(","))
    _, _, err = S.sphdvr_lut_build("m4", K, D, 257)
    E = S.sphdvr_lut_error_measure("m4", err)
    assert abs(E / table["E"][key] - 1) < 1.5e-4


def test_lut_error_measure_special_cases():
    # poly6 is a polynomial in r^2: its ray restriction is represented exactly for D = 6
    _, _, err = S.sphdvr_lut_build("poly6", 1, 6, 33)
    assert S.sphdvr_lut_error_measure("poly6", err) < 1e-9
    # a constant per-entry error e gives e * sqrt(pi q^2) / kappa (closed form of the Lambda integral)
    kap = math.sqrt(4 * math.pi * quad(lambda r: (r * oracle.kernel_w("wendland_c2", r)) ** 2, 0, 2, epsabs=1e-16)[0])
    for n in (65, 64):
        E = S.sphdvr_lut_error_measure("wendland_c2", np.full(n, 1e-3))
        assert abs(E / (1e-3 * math.sqrt(math.pi * 4.0) / kap) - 1) < 1e-9
    for bad in (np.zeros(2), np.array([0.0, -1.0, 0.0]), np.array([0.0, np.nan, 0.0])):
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_lut_error_measure("m4", bad)
        assert e.value.status == S.EINVAL


@pytest.mark.parametrize("D", [2, 3, 4, 5, 6])
def test_quant_params_reproduce_the_printed_quantisation_errors(D):
    """sphdvr_quant_params gives the paper's printed Q_E bars (Sec. 5.2 figure: M4, 64 bits, ratio 1e5)."""
    g = json.load(open(os.path.join(HERE, "golden", "paper_quant_error.json")))
    tau, sigma, qe = S.sphdvr_quant_params(g["kernel"], D, g["int_bits"], g["variance_ratio"])
    assert abs(qe / g["QE"][str(D)] - 1) < 1e-12
    assert abs(S.sphdvr_quant_error(g["kernel"], D, tau, sigma) / qe - 1) < 1e-15


def test_combined_error_from_the_library_matches_the_printed_marks():
    g = json.load(open(os.path.join(HERE, "golden", "paper_quant_error.json")))
    for key in ("4,3", "3,2", "2,5", "4,4"):
        K, D = map(int, key.split(","))
        _, _, err = S.sphdvr_lut_build("m4", K, D, 257)
        E = S.sphdvr_lut_error_measure("m4", err)
        qe = S.sphdvr_quant_params("m4", D, 64, 1e5)[2]
        assert abs(math.sqrt(E * E + qe * qe) / g["combined"][key] - 1) < 1.5e-4


@pytest.mark.parametrize("kernel", ["wendland_c2", "wendland_c4", "poly6"])
def test_quant_error_agrees_with_the_oracle(kernel):
    from oracle import quant as OQ

    for D, bits, ratio in ((1, 32, 10.0), (3, 64, 1e5), (5, 96, 1e3)):
        t_l, s_l, q_l = S.sphdvr_quant_params(kernel, D, bits, ratio)
        t_o, s_o, q_o = OQ.quant_params(kernel, D, bits, ratio)
        assert abs(t_l / t_o - 1) < 1e-12 and abs(s_l / s_o - 1) < 1e-14 and abs(q_l / q_o - 1) < 1e-12
        assert abs(S.sphdvr_quant_error(kernel, D, 3 * t_o, s_o) / OQ.quant_error(kernel, D, 3 * t_o, s_o) - 1) < 1e-12


def test_quant_functions_reject_bad_arguments():
    for args in (("m4", 3, 0.0, 1e-9), ("m4", 3, -1.0, 1e-9), ("m4", -1, 1e-3, 1e-9), ("m4", 3, 1e-3, -1.0),
                 (7, 3, 1e-3, 1e-9), ("m4", 3, float("nan"), 1e-9)):
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_quant_error(*args)
        assert e.value.status == S.EINVAL
    for args in (("m4", 3, 4, 1e5), ("m4", 3, 64, 0.0), ("m4", 3, 64, -1.0), (9, 3, 64, 1e5)):
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_quant_params(*args)
        assert e.value.status == S.EINVAL


def test_table_file_roundtrip_and_malformed_files(tmp_path):
    """sphdvr_lut_save / sphdvr_lut_read give back the built table bit for bit; bad files are refused."""
    th, pc, err = S.sphdvr_lut_build("m4", 3, 2, 33)
    path = str(tmp_path / "m4_K3_D2.lut")
    S.sphdvr_lut_save(path, "m4", 3, 2, 33, th, pc, err)
    k, K, D, n, th2, pc2, err2 = S.sphdvr_lut_read(path)
    assert (k, K, D, n) == (oracle.KERNELS["m4"], 3, 2, 33)
    assert np.array_equal(th2, th) and np.array_equal(pc2, pc) and np.array_equal(err2, err)
    raw = open(path, "rb").read()
    assert len(raw) == 40 + 8 * (33 * 2 + 33 * 2 * 3 + 33)
    cases = {"magic": b"X" + raw[1:], "short": raw[:-8], "trailing": raw + b"\0",
             "bad_K": raw[:16] + (9).to_bytes(4, "little") + raw[20:]}
    for name, data in cases.items():
        bad = str(tmp_path / (name + ".lut"))
        open(bad, "wb").write(data)
        with pytest.raises(S.SphdvrError) as e:
            S.sphdvr_lut_read(bad)
        assert e.value.status == S.EINVAL, name
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_lut_read(str(tmp_path / "missing.lut"))
    assert e.value.status == S.ENOTFOUND
    with pytest.raises(S.SphdvrError) as e:
        S.sphdvr_lut_save(path, "m4", 9, 2, 33, th, pc, err)
    assert e.value.status == S.EINVAL


def test_header_is_plain_c(tmp_path):
    """include/sphdvr.h is a C ABI: it compiles as pedantic C99 (and as C++)."""
    import subprocess

    src = tmp_path / "h.c"
    src.write_text('#include "sphdvr.h"\nint main(void) { return SPHDVR_OK + SPHDVR_MAX_BATCH - 8; }\n')
    inc = os.path.join(os.path.dirname(HERE), "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", inc, str(src)],
                   check=True)
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Werror", "-fsyntax-only", "-I", inc, "-x", "c++", str(src)],
                   check=True)


@pytest.mark.parametrize("kernel,K,D", [("m4", 4, 3), ("wendland_c2", 4, 3), ("m4", 3, 2), ("poly6", 1, 6)])
def test_library_gradient_table_matches_the_oracle(kernel, K, D):
    """The library's gradient builder (host, long double) and the oracle's (FP64) project the same
    G_L = w'(rho)/rho on the same knots: the pieces agree to rounding, relative to the entry's norm of G."""
    n = 65
    L = oracle.lut_build(kernel, K, D, n)
    G = oracle.lut_build_grad(L)
    gp, ge = S.sphdvr_lut_build_grad(kernel, K, D, n, L["theta"])
    for j in range(n - 1):
        scale = max(G["normG"][j], 1e-300)
        assert np.abs(gp[j] - G["gpieces"][j]).max() <= 1e-9 * scale
        assert abs(ge[j] - G["gerr"][j]) <= 1e-12 * scale
    assert np.all(gp[-1] == 0)
    with pytest.raises(S.SphdvrError):
        S.sphdvr_lut_build_grad(kernel, K, 9, n, L["theta"])
