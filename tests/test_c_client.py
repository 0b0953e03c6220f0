"""The C ABI from plain C: include/nbcluster.h compiles as strict C99 on its
own, and a C program linked against the library gets the same results from
the host-only entry points as the Python binding (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

import paper_1306_1737_gb300 as nb
from paper_1306_1737_gb300 import build as nbbuild

HERE = os.path.dirname(os.path.abspath(__file__))
INCLUDE = os.path.join(os.path.dirname(HERE), "include")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    lib = nbbuild.build()
    out = str(tmp_path_factory.mktemp("c_client") / "client")
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INCLUDE,
                    os.path.join(HERE, "c_client", "client.c"), "-o", out, "-L", libdir, "-lnbcluster",
                    f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([out], capture_output=True, text=True, check=True)
    return {ln.split()[0]: ln.split()[1:] for ln in r.stdout.splitlines()}


def test_header_is_strict_c99(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "h.c"
    src.write_text('#include "nbcluster.h"\nint main(void) { return NB_OK; }\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-I", INCLUDE,
                    str(src)], check=True)


def test_c_client_matches_the_binding(client):
    import numpy as np
    t = nb.nb_lj_combine([0.3166, 0.0], [0.650, 0.0])
    assert client["lj"][0] == "0"
    assert float(client["lj"][1]) == pytest.approx(float(t[0, 0, 0]), rel=1e-7)
    assert float(client["lj"][2]) == pytest.approx(float(t[0, 0, 1]), rel=1e-7)
    assert client["plan"] == ["0", str(nb.nb_workspace_bytes(8, 24000, [6.21] * 3, 1.1, 2))]
    assert client["refused"] == [str(nb.NB_ERR_CAPACITY), "NB_ERR_CAPACITY"]
    cls = [(8000, 15.9994, -0.82, 0), (16000, 1.008, 0.41, 1)]
    p = nb.make_params("ewald", 1.0, beta=3.12, want_energy=False)
    vol = 6.21 ** 3
    drift = nb.nb_buffer_drift(cls, t, vol, p, 0.1, 0.038, 300.0)
    assert client["drift"][0] == "0" and float(client["drift"][1]) == pytest.approx(drift, rel=1e-12)
    rb = nb.nb_buffer_size(cls, t, vol, p, 0.038, 300.0, 0.00249)
    assert client["size"][0] == "0" and float(client["size"][1]) == pytest.approx(rb, abs=2e-9)
    assert np.isfinite(drift) and drift > 0 and 0 < rb < 1
    assert client["frames"] == [str(nb.NB_ERR_ARG), "NB_ERR_ARG"]
