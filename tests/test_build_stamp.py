"""build() reuses a built library only under the source hash it was built from (CPU only)."""
import pytest

from paper_2604_22228_gb300 import build


class _Compiled(Exception):
    pass


def _no_compile(nvcc, src):
    raise _Compiled(src)


def test_hash_tracks_sources_flags_and_compiler(monkeypatch):
    h = build.source_hash("/usr/local/cuda/bin/nvcc")
    assert h == build.source_hash("/usr/local/cuda/bin/nvcc")
    assert h != build.source_hash("/other/nvcc")
    monkeypatch.setattr(build, "CFLAGS", build.CFLAGS + ["-DMPT_SOMETHING_ELSE"])
    assert h != build.source_hash("/usr/local/cuda/bin/nvcc")


def test_reuse_needs_a_matching_stamp(monkeypatch, tmp_path):
    out = tmp_path / "libmpt.so"
    stamp = tmp_path / "libmpt.so.sha256"
    out.write_bytes(b"not a library")
    monkeypatch.setattr(build, "OUT", str(out))
    monkeypatch.setattr(build, "STAMP", str(stamp))
    monkeypatch.setattr(build, "OBJDIR", str(tmp_path / "obj"))
    monkeypatch.setattr(build, "_compile", _no_compile)
    nvcc = build._nvcc()
    # no stamp (a library shipped or copied in without one): rebuild
    with pytest.raises(_Compiled):
        build.build()
    # a stamp of other sources: rebuild
    stamp.write_text("0" * 64 + "\n")
    with pytest.raises(_Compiled):
        build.build()
    # the current sources' stamp: reuse without compiling
    stamp.write_text(build.source_hash(nvcc) + "\n")
    assert build.build() == str(out)
    # force: always rebuild
    with pytest.raises(_Compiled):
        build.build(force=True)
