"""The checkpoint writer's host path against the documented format (no GPU needed).

A small host program (tests/ckpt_writer_host.cpp) drives ns::CkptWriter; the file it
leaves must carry the magic, the record, the payload and the word-wise FNV-1a
checksum, be accepted by ns_read_checkpoint, and replace the previous file only on
commit (an abandoned write leaves the old file and no temporary behind).
"""

import os
import shutil
import struct
import subprocess

import pytest

from test_checkpoint_format import fnv1a_words

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def writer(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ and the CUDA headers are needed to build the writer driver")
    exe = str(tmp_path_factory.mktemp("w") / "ckpt_writer_host")
    cmd = [gxx, "-std=c++17", "-O1", "-I", os.path.join(CUDA, "include"), os.path.join(HERE, "ckpt_writer_host.cpp"),
           "-o", exe, "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr[-2000:])
    return exe


@pytest.fixture
def ns(lib):
    from paper_2407_04634_gb300 import nullspace
    return nullspace


@pytest.mark.parametrize("length", [0, 5, 64, 1 << 20])
def test_committed_file_follows_the_format(writer, ns, tmp_path, length):
    path = str(tmp_path / "a.ckpt")
    assert subprocess.run([writer, path, "commit", str(length)]).returncode == 0
    raw = open(path, "rb").read()
    assert raw[:8] == b"NSCKPT01"
    body, tail = raw[:-8], raw[-8:]
    assert struct.unpack("<Q", tail)[0] == fnv1a_words(body)
    payload = body[8 + 184:]
    assert payload == bytes((i * 37 + 11) & 0xFF for i in range(length))
    info = ns.read_checkpoint(path)
    assert info["restarts"] == length and info["k0"] == 4 and info["seed"] == 77
    assert not os.path.exists(path + ".tmp")


def test_abandoned_write_keeps_the_previous_file(writer, ns, tmp_path):
    path = str(tmp_path / "b.ckpt")
    assert subprocess.run([writer, path, "commit", "100"]).returncode == 0
    before = open(path, "rb").read()
    assert subprocess.run([writer, path, "abandon", "5000"]).returncode == 0
    assert open(path, "rb").read() == before
    assert not os.path.exists(path + ".tmp")
    assert ns.read_checkpoint(path)["restarts"] == 100


def test_unwritable_path_is_refused(writer, tmp_path):
    assert subprocess.run([writer, str(tmp_path / "no" / "such" / "dir.ckpt"), "commit", "8"]).returncode == 3
