"""The apply launch-shape tuner's persistent cache (ASM_TUNE_CACHE)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def P():
    from paper_2401_03915_gb300 import build
    build.build()
    import paper_2401_03915_gb300 as P
    P.load()
    return P


def test_apply_tuner_cache_file(P, tmp_path):
    """With ASM_TUNE_CACHE set, the apply tuner writes its choice for a shape
    to the file once; a later process reads it instead of timing again (no
    second line)."""
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.jsonl"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); import paper_2401_03915_gb300 as P; P.load(); "
            "from asm_inputs import diffusion3d; p = diffusion3d(12, (2, 2, 2), contrast=1e3, nev=4); "
            "S = P.TwoLevelSchwarz(p.indptr, p.indices, p.data, p.part, p.N, 1, 4, precision='fp32'); S.close()" % root)
    env = dict(os.environ, ASM_TUNE_CACHE=str(path))
    for _ in range(2):
        subprocess.run([sys.executable, "-c", code], env=env, cwd=root, check=True, timeout=600)
    lines = path.read_text().splitlines()
    assert len(lines) == 1, lines
    assert '"tile_ctas": ' in lines[0] and '"device": ' in lines[0]
