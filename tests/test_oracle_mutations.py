"""Planted mistakes in the CPU oracle: each one must fail at least one of its pins.

A pin is only worth something if a plausible slip in the code it guards makes it fail.  For every entry below, a
temporary copy of the repository gets the oracle with one mistake planted -- a dropped term, a wrong sign, index or
boundary, a swapped operand or conjugate, a wrong scale -- and the oracle's CPU pins (``tests/test_oracle*.py``) run
there in a separate process; the test passes when every planted mistake makes that run fail.  Nothing here touches
a GPU or the CUDA library."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle", "nlinv_oracle.py")
PINS = ["tests/test_oracle.py", "tests/test_oracle_newton.py", "tests/test_oracle_properties.py"]

# (what is planted, oracle text, planted text)
MISTAKES = [
    ("Nyquist index on the wrong side", "return (i + n // 2) % n - n // 2", "return (i + n // 2 - 1) % n - n // 2 + 1"),
    ("Sobolev exponent -l instead of -l/2", "** (-l / 2.0)", "** (-l)"),
    ("frequency scaled by n - 1", "k = signed_index(n) / n", "k = signed_index(n) / (n - 1)"),
    ("Omega boundary shifted", "((g >= -fov) & (g < fov))", "((g > -fov) & (g <= fov))"),
    ("FFT not unitary", 'return np.fft.fft2(a, axes=(-2, -1), norm="ortho")', "return np.fft.fft2(a, axes=(-2, -1))"),
    ("scalar product conjugates the second argument", "np.vdot(u.ravel(), v.ravel())", "np.vdot(v.ravel(), u.ravel())"),
    ("W^-1 with the forward transform", "return ifft2u(sobolev_weight(s.n, s.a, s.l) * chat)",
     "return fft2u(sobolev_weight(s.n, s.a, s.l) * chat)"),
    ("W^-H with the inverse transform", "return sobolev_weight(s.n, s.a, s.l) * fft2u(u)",
     "return sobolev_weight(s.n, s.a, s.l) * ifft2u(u)"),
    ("channel sum conjugates the data", "np.sum(np.conj(c) * z, axis=0)", "np.sum(c * np.conj(z), axis=0)"),
    ("F without M_Omega", "return mask * fft2u(M * x[0] * c)", "return mask * fft2u(x[0] * c)"),
    ("DF with a sign flip", "fft2u(M * (dx[0] * c + x[0] * dc))", "fft2u(M * (dx[0] * c - x[0] * dc))"),
    ("DF with drho in place of rho", "fft2u(M * (dx[0] * c + x[0] * dc))", "fft2u(M * (dx[0] * c + dx[0] * dc))"),
    ("DF^H without conj(rho)", "out[1:] = WiH(s, np.conj(x[0]) * z)", "out[1:] = WiH(s, x[0] * z)"),
    ("DF^H without M_Omega", "z = M * ifft2u(mask * r)", "z = ifft2u(mask * r)"),
    ("normal operator minus alpha", "return adjoint(s, mask, x, derivative(s, mask, x, d, c), c) + alpha * d",
     "return adjoint(s, mask, x, derivative(s, mask, x, d, c), c) - alpha * d"),
    ("simulated data without M_Omega", "return mask * fft2u(M * rho * coil_img)", "return mask * fft2u(rho * coil_img)"),
    ("gridding samples shifted by one", "t = -n / 2 + 0.5 * i", "t = -n / 2 + 0.5 * (i + 1)"),
    ("gridding rounds half to even", "kx = int(np.floor(t * np.cos(th) + 0.5))", "kx = int(np.round(t * np.cos(th)))"),
    ("gridding sums instead of averaging", "y[:, hit] = total[:, hit] / count[hit]", "y[:, hit] = total[:, hit]"),
    ("gridding with the axes swapped", "total[:, ky % n, kx % n] += samples[:, si, i]",
     "total[:, kx % n, ky % n] += samples[:, si, i]"),
    ("image without the square root", "full = x[0] * np.sqrt(np.sum(np.abs(coils(s, x)) ** 2, axis=0))",
     "full = x[0] * np.sum(np.abs(coils(s, x)) ** 2, axis=0)"),
    ("image cropped one pixel off", "return shifted[h - s.fov: h + s.fov, h - s.fov: h + s.fov]",
     "return shifted[h - s.fov + 1: h + s.fov + 1, h - s.fov + 1: h + s.fov + 1]"),
    ("CG beta inverted", "beta = rr_new / rr", "beta = rr / rr_new"),
    ("CG residual updated with p", "r = r - a * q", "r = r - a * p"),
    ("CG floor absolute", "if not (rr > floor2 * rr0 and np.isfinite(rr)):", "if not (rr > floor2 and np.isfinite(rr)):"),
    ("CG floor at 2^-12 instead of 2^-24", "CG_FLOOR2 = 2.0 ** -48", "CG_FLOOR2 = 2.0 ** -24"),
    ("residual norm squared", "return r, float(np.sqrt(inner(r, r).real))", "return r, float(inner(r, r).real)"),
    ("alpha schedule starts at alpha_0 q", "alpha0 * q ** k", "alpha0 * q ** (k + 1)"),
    ("alpha floor ignored", "[max(alpha0 * q ** k, alpha_min)", "[(alpha0 * q ** k)"),
    ("single frame regularised toward zero", "xr = x.copy() if xref is None else np.asarray(xref, dtype=np.complex128)",
     "xr = np.zeros_like(x) if xref is None else np.asarray(xref, dtype=np.complex128)"),
    ("regulariser sign flipped", "b = adjoint(s, mask, x, r0, c) - alpha * (x - xr)",
     "b = adjoint(s, mask, x, r0, c) + alpha * (x - xr)"),
    ("regulariser without x_ref", "b = adjoint(s, mask, x, r0, c) - alpha * (x - xr)",
     "b = adjoint(s, mask, x, r0, c) - alpha * x"),
    ("gradient to x_ref without alpha", "gref = gref + alpha * u", "gref = gref + u"),
    ("gradient's second term sign", "g = adjoint(s, mask, u, sres) - adjoint(s, mask, dx, v)",
     "g = adjoint(s, mask, u, sres) + adjoint(s, mask, dx, v)"),
    ("gradient's residual without DF dx", "sres = y - forward(s, mask, x) - derivative(s, mask, x, dx, c)",
     "sres = y - forward(s, mask, x)"),
    ("series regularised toward the first start value",
     "prev, _ = irgnm(s, mask, y, prev, prev, newton_steps, cg_iters, alpha0, q, alpha_min)",
     "prev, _ = irgnm(s, mask, y, prev, x0, newton_steps, cg_iters, alpha0, q, alpha_min)"),
]


@pytest.fixture(scope="module")
def sandbox(tmp_path_factory):
    root = tmp_path_factory.mktemp("oracle_mutations")
    skip = shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.o")
    for d in ("oracle", "tests", "paper_1301_1215_gb300"):
        shutil.copytree(os.path.join(ROOT, d), root / d, ignore=skip)
    return root


def test_unmutated_oracle_passes_its_pins(sandbox):
    shutil.copy(ORACLE, sandbox / "oracle" / "nlinv_oracle.py")
    r = _run_pins(sandbox)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("what,text,planted", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(sandbox, what, text, planted):
    src = open(ORACLE).read()
    assert src.count(text) >= 1, f"the oracle no longer contains the text this entry mutates: {text!r}"
    (sandbox / "oracle" / "nlinv_oracle.py").write_text(src.replace(text, planted))
    r = _run_pins(sandbox)
    assert r.returncode != 0, f"no pin fails with: {what}"


def _run_pins(root):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider"] + PINS,
                          cwd=root, capture_output=True, text=True, env=env, timeout=600)
