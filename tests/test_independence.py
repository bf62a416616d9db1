"""Separation of the oracle from the product, checked on the sources (CPU only): the library
package never imports the oracle (no route from the product path into test infrastructure), the
oracle imports nothing from the package (it shares no code with the CUDA path), and the seeded
input generators import neither (they hold no arithmetic of the method)."""
import ast
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2402_02116_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name for a in node.names}
        elif isinstance(node, ast.ImportFrom):
            mods.add(("." * node.level) + (node.module or ""))
    return mods


def py_files(folder):
    return [os.path.join(folder, f) for f in sorted(os.listdir(folder)) if f.endswith(".py")]


def test_the_package_never_imports_the_oracle():
    for path in py_files(PKG):
        bad = {m for m in imported_modules(path) if m == "oracle" or m.startswith("oracle.")}
        assert not bad, (path, bad)
    for name in os.listdir(os.path.join(PKG, "csrc")):
        for line in open(os.path.join(PKG, "csrc", name)):
            assert not (line.lstrip().startswith("#include") and "oracle" in line), (name, line)


def test_the_oracle_imports_nothing_from_the_package():
    for path in py_files(ORACLE):
        bad = {m for m in imported_modules(path) if "paper_2402_02116_gb300" in m}
        assert not bad, (path, bad)


def test_the_input_generators_import_neither():
    mods = imported_modules(os.path.join(PKG, "inputs.py"))
    assert not any(m.startswith("oracle") or m.startswith(".") or "paper_2402_02116_gb300" in m for m in mods), mods


def test_the_cpp_oracle_includes_nothing_from_the_library():
    """The C++ oracle's sources include only the standard library (and OpenMP): no header of the
    CUDA library, no CUDA runtime."""
    folder = os.path.join(ORACLE, "cpp")
    for name in os.listdir(folder):
        if not name.endswith((".cpp", ".h", ".hpp")):
            continue
        for line in open(os.path.join(folder, name)):
            if line.lstrip().startswith("#include"):
                inc = line.split("#include", 1)[1].strip()
                assert inc.startswith("<") and "cuda" not in inc and "dbi" not in inc, (name, line)
