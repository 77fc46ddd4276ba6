"""The oracle's pins catch plausible mistakes.  Each mutant below plants one
error in a copy of the oracle (its C core or its Python finalize / PCE: a
wrong sign, index, radius, reduction, constant or dropped term); the copy is
built with gcc and the pin files tests/test_oracle_{wavelet,denoise,
sda_mle_pce}.py (tests/test_oracle_grad.py for the adjoints of grad.py) run
against it in a subprocess: at least one pin must fail.
The unmutated copy, run the same way, must pass (so a broken harness cannot
look like a caught mutant).  CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["test_oracle_wavelet.py", "test_oracle_denoise.py", "test_oracle_sda_mle_pce.py"]
GRAD_PIN_FILES = ["test_oracle_grad.py"]

# name, oracle file, text (must occur exactly once in it), replacement
MUTANTS = [
    ("highpass taps not reversed", "prnu_oracle.c", "* h[L - 1 - k];", "* h[k];"),
    ("analysis index sign", "prnu_oracle.c", "double v = x[wrap_index(2L * n + k, N) * xs];",
     "double v = x[wrap_index(2L * n - k, N) * xs];"),
    ("window radius off by one", "prnu_oracle.c", "int w = windows[wi], rad = w / 2;",
     "int w = windows[wi], rad = w / 2 + 1;"),
    ("max over windows instead of min", "prnu_oracle.c", "if (mean < vmin) vmin = mean;",
     "if (mean > vmin || vmin == INFINITY) vmin = mean;"),
    ("sigma0 used for sigma0^2", "prnu_oracle.c", "double s2 = sigma0 * sigma0;", "double s2 = sigma0;"),
    ("noise details in the denoised image", "prnu_oracle.c",
     "rc = orc_idwt2_level(rec, cleanD[l][0], cleanD[l][1], cleanD[l][2], R, Cc, h, L, tmp);",
     "rc = orc_idwt2_level(rec, noiseD[l][0], cleanD[l][1], cleanD[l][2], R, Cc, h, L, tmp);"),
    ("mirror without edge repeat", "prnu_oracle.c", "return i < n ? i : 2 * n - 1 - i;",
     "return i < n ? i : 2 * n - 2 - i;"),
    ("MLE numerator W.W", "prnu_oracle.c", "num[i] += Wr[i] * I[i];", "num[i] += Wr[i] * Wr[i];"),
    ("ragged group divided by d", "prnu_oracle.c",
     "out[(((long)i * C + c) * H + y) * W + x] = (double)s / (double)n;",
     "out[(((long)i * C + c) * H + y) * W + x] = (double)s / (double)d;"),
    ("LL4 dropped from the denoised image", "prnu_oracle.c", "memcpy(rec, LLs[levels], n * sizeof(double));",
     "memset(rec, 0, n * sizeof(double));"),
    ("variance floor without sigma0^2", "prnu_oracle.c", "double var = vmin - s2 > 0.0 ? vmin - s2 : 0.0;",
     "double var = vmin > 0.0 ? vmin : 0.0;"),
    ("correlation conjugates the wrong operand", "pipeline.py",
     "np.conj(np.fft.fft2(X)) * np.fft.fft2(Y)", "np.fft.fft2(X) * np.conj(np.fft.fft2(Y))"),
    ("PCE query mean kept", "pipeline.py", "    Y = Y - Y.mean()\n", ""),
    ("PCE neighbourhood one smaller", "pipeline.py", "    r = nbhd // 2\n", "    r = nbhd // 2 - 1\n"),
    ("PCE unsigned", "pipeline.py", "pce = np.sign(c0) * c0 * c0 / energy", "pce = c0 * c0 / energy"),
    ("PCE energy summed, not averaged", "pipeline.py", "energy = float(np.mean(C[mask] ** 2))",
     "energy = float(np.sum(C[mask] ** 2))"),
    ("grey weights of R and B swapped", "pipeline.py",
     "GRAY_WEIGHTS[0] * x[0] + GRAY_WEIGHTS[1] * x[1] + GRAY_WEIGHTS[2] * x[2]",
     "GRAY_WEIGHTS[2] * x[0] + GRAY_WEIGHTS[1] * x[1] + GRAY_WEIGHTS[0] * x[2]"),
    ("zero-mean over rows only", "pipeline.py", "    K = K - K.mean(axis=0, keepdims=True)\n", ""),
    ("Wiener noise level as std", "pipeline.py", "sig2 = float(np.var(K))", "sig2 = float(np.std(K))"),
    ("Wiener magnitude not normalised", "pipeline.py", "M = np.abs(F) / np.sqrt(N)", "M = np.abs(F)"),
    # adjoints (pinned by tests/test_oracle_grad.py).  Not listed: dropping the
    # mean removal of the PCE adjoint, which is equivalent (the correlation of
    # G with the zero-mean Y already has zero mean).
    ("shrink adjoint without the argmin-window term", "grad.py", "gc = gc + 2.0 * c * _box_sum(a, w)",
     "gc = gc + 0.0 * c * _box_sum(a, w)"),
    ("shrink adjoint without d(s0^2)/d(s0)", "grad.py", "return gc, 2.0 * sigma0 * g_s2", "return gc, g_s2"),
    ("MLE adjoint of den halved", "grad.py", "g_num[None] * Wr + 2.0 * g_den[None] * S",
     "g_num[None] * Wr + g_den[None] * S"),
    ("PCE adjoint correlates where it convolves", "grad.py",
     "gYc = np.real(np.fft.ifft2(np.fft.fft2(X) * np.fft.fft2(G)))",
     "gYc = np.real(np.fft.ifft2(np.conj(np.fft.fft2(X)) * np.fft.fft2(G)))"),
    ("SDA weight adjoint from the wrong group", "grad.py", "float(np.sum(gS[j // d] * np.transpose",
     "float(np.sum(gS[(j + 1) // d % gS.shape[0]] * np.transpose"),
]


def _run_pins(tmp_path, replace=None) -> subprocess.CompletedProcess:
    """Copy the oracle (with `replace` = (file, text) substituted), the pin
    files and what they import into tmp_path, and run the pins there."""
    (tmp_path / "tests").mkdir()
    (tmp_path / "paper_1909_04573_gb300").mkdir()
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.so.*", "__pycache__"))
    if replace:
        (tmp_path / "oracle" / replace[0]).write_text(replace[1])
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    for f in ["conftest.py"] + PIN_FILES + GRAD_PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    for f in ["__init__.py", "synth.py"]:
        shutil.copy(os.path.join(ROOT, "paper_1909_04573_gb300", f), tmp_path / "paper_1909_04573_gb300" / f)
    env = dict(os.environ, PYTHONPATH=str(tmp_path), PYTHONDONTWRITEBYTECODE="1")
    files = GRAD_PIN_FILES if replace and replace[0] == "grad.py" else PIN_FILES
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                          [os.path.join("tests", f) for f in files],
                          cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)


def _source(name):
    with open(os.path.join(ROOT, "oracle", name)) as f:
        return f.read()


def test_unmutated_copy_passes_the_pins(tmp_path):
    r = _run_pins(tmp_path)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    # and the adjoint pins, on an unchanged copy of grad.py
    (tmp_path / "g").mkdir()
    r = _run_pins(tmp_path / "g", ("grad.py", _source("grad.py")))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.mark.parametrize("name,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(tmp_path, name, fname, old, new):
    src = _source(fname)
    assert src.count(old) == 1, f"mutation site of '{name}' not unique in {fname}"
    r = _run_pins(tmp_path, (fname, src.replace(old, new)))
    assert r.returncode == 1, f"'{name}' not caught (pytest exit {r.returncode}):\n" + r.stdout[-1500:]
    assert "failed" in r.stdout
