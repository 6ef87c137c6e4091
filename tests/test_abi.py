"""The C ABI library loads and exports every symbol include/spfom.h declares
(CPU only: no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spfom.h")
HEADERS = [os.path.join(ROOT, "include", f) for f in ("spfom.h", "spfom_mlp.h")]


@pytest.fixture(scope="module")
def libpath():
    from paper_2602_22421_gb300.build import build
    return build()


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(spfom_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_api():
    names = declared_functions()
    for want in ("spfom_create", "spfom_load_instance", "spfom_step", "spfom_solve", "spfom_duals"):
        assert want in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(spfom_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    import paper_2602_22421_gb300 as pkg
    assert sorted(pkg.EXPORTS) == declared_functions()
    h = pkg.lib()
    for f in declared_functions():
        assert hasattr(h, f)


def test_defaults_and_status_strings(libpath):
    import paper_2602_22421_gb300 as pkg
    p = pkg.default_params()
    assert (p.precision, p.tau, p.tau0, p.mu, p.batch_frac, p.eval_every) == (64, 0.0, 0.1, 0.0, 1.0, 64)
    assert (p.restart_beta, p.restart_artificial, p.restart_tau_decay, p.kkt_tol) == (0.2, 0.36, 1.0, 1e-4)
    h = pkg.lib()
    assert h.spfom_status_string(0) == b"SPFOM_OK"
    assert h.spfom_status_string(7) == b"SPFOM_ENOTSUP"
    assert h.spfom_last_error(None) == b"ctx is NULL"


def test_create_without_gpu_fails_cleanly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2602_22421_gb300 as pkg
    with pytest.raises(pkg.SpfomError) as ei:
        pkg.Solver()
    assert ei.value.status == 3  # SPFOM_ECUDA


def test_struct_layouts_match_header():
    """The ctypes mirrors list the header's struct fields in order."""
    import paper_2602_22421_gb300.spfom as b
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)

    def fields(struct):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + ";", text).group(1)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            decl = re.sub(r"\[[^\]]*\]", "", decl)
            parts = decl.split()
            rest = " ".join(parts[1:]) if not decl.startswith("const") else " ".join(parts[2:])
            names += [x.strip(" *") for x in rest.split(",")]
        return names

    assert fields("spfom_params") == [f for f, _ in b.Params._fields_]
    assert fields("spfom_instance") == [f for f, _ in b.InstanceC._fields_]
    assert fields("spfom_stats") == [f for f, _ in b.Stats._fields_]
    assert fields("spfom_device_segments") == [f for f, _ in b.DeviceSegments._fields_]
    assert re.search(r"#define SPFOM_NOALLOC_MAX_PRODUCTS (\d+)", text).group(1) == str(b.NOALLOC_MAX_PRODUCTS)
