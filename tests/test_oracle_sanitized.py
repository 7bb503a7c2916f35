"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

The oracle's C sources are rebuilt with -fsanitize=address,undefined (no recovery)
into a scratch directory, and a child process with the ASan runtime preloaded
drives that build through small gradients that touch every code path of the
oracle: the steady and unsteady 2-D channel, the thermal lattice with the heat
source, the Boussinesq force and a heated wall segment, the pressure-drop and
energy-loss objectives, the periodic mode, and the 3-D duct.  Any out-of-bounds
access or undefined behaviour aborts the child, which fails the test.
"""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    from oracle import oracle as O
    O._LIB = {lib!r}   # the sanitized build (newer than the sources, so not rebuilt)
    import inputs

    def grad2(pb, g=None):
        g = pb.gamma() if g is None else g
        return O.steady_gradient(pb, g) if pb.steady else O.unsteady_gradient(pb, g)

    base = dict(seed=1, sigma=2.0, strip=2, n_steps=25, n_adj=25)
    grad2(inputs.channel(20, 12, Re=10.0, **base))
    grad2(inputs.channel(20, 12, Re=10.0, kappa_p=1.0, kappa_E=1.0, **base))
    grad2(inputs.channel(20, 12, Re=10.0, steady=False, pulse_mean=0.75, pulse_amp=0.25,
                         pulse_period=10.0, kappa_E=1.0, **base))
    th = inputs.channel(20, 12, Re=10.0, thermal=1, kappa_T=1e-2, t_kind=[0, 1, 0, 1],
                        t_val=[0.0, 0.0, 1.0, 0.0], beta_bar=0.01, kappa_Q=1.0, gb_y=-1e-3,
                        steady=False, pulse_mean=0.75, pulse_amp=0.25, pulse_period=10.0, **base)
    th.K_f = th.nu / 0.71
    th.K_s = th.K_f
    grad2(th)
    pb, g = inputs.natural_convection_cavity(scale=0.2)
    O.steady_gradient(pb.with_(n_steps=20, n_adj=20), g)
    grad2(inputs.channel(20, 12, Re=10.0, periodic=1, G_x=1e-5, **base))
    d3 = inputs.duct(9, 7, 8, Re=5.0, seed=7, sigma=2.0, strip=2, n_steps=10, n_adj=10, kappa_p=1.0)
    O.steady_gradient3(d3, d3.gamma())
    print("oracle clean")
""")


def _runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_oracle_runs_clean_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    asan = _runtime("libasan.so")
    if asan is None:
        pytest.skip("no AddressSanitizer runtime for gcc")
    lib = str(tmp_path / "liblks_oracle_san.so")
    src = [os.path.join(ROOT, "oracle", "lks_oracle.c"), os.path.join(ROOT, "oracle", "lks3d_oracle.c")]
    subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
                    "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer",
                    "-o", lib, *src, "-lm"], check=True)
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, lib=lib)], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "oracle clean" in r.stdout, r.stderr[-6000:]
