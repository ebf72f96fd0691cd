"""Host-side checks of the checkpoint file format (no GPU needed).

A checkpoint is: the magic "NSCKPT01", the ns_checkpoint_info record, the solver
state, and a 64-bit FNV-1a checksum of everything before it, taken over
little-endian 64-bit words with a zero-padded tail.  The files here are written by
this test from that description alone, so the reader in the library is checked
against the documented format, not against its own writer.
"""

import ctypes
import struct

import pytest

FNV_OFFSET = 14695981039346656037
FNV_PRIME = 1099511628211


def fnv1a_words(data: bytes) -> int:
    if len(data) % 8:
        data = data + b"\0" * (8 - len(data) % 8)
    h = FNV_OFFSET
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    return h


def record(ns, **kw):
    r = ns.NsCheckpointInfo()
    vals = dict(version=1, m=5, n=4, nnz=9, mode=0, precision=0, d=2, restart_len=12, reorth=0, gemm=0,
                fp64_products=0, spmm_A=8, spmm_At=4, seed=77, eps=1e-3, tol_eff=1e-10, normA1=3.5, normAinf=2.25,
                matvecs=48, restarts=2, nullity=1, k0=4, precond=0.0)
    vals.update(kw)
    for k, v in vals.items():
        setattr(r, k, v)
    return bytes(r)


def write(tmp_path, body: bytes, name="c.ckpt", checksum=None):
    p = tmp_path / name
    c = fnv1a_words(body) if checksum is None else checksum
    p.write_bytes(body + struct.pack("<Q", c))
    return p


@pytest.fixture
def ns(lib):
    from paper_2407_04634_gb300 import nullspace
    return nullspace


def test_record_layout_is_all_eight_byte_fields(ns):
    assert ctypes.sizeof(ns.NsCheckpointInfo) == 8 * len(ns.NsCheckpointInfo._fields_) == 8 * 23


@pytest.mark.parametrize("payload_len", [0, 8, 13, 1000])
def test_reads_a_file_written_from_the_format(ns, tmp_path, payload_len):
    body = b"NSCKPT01" + record(ns) + bytes(range(256)) * (payload_len // 256) + bytes(payload_len % 256)
    info = ns.read_checkpoint(write(tmp_path, body))
    assert info["n"] == 4 and info["m"] == 5 and info["d"] == 2 and info["restart_len"] == 12
    assert info["seed"] == 77 and info["eps"] == 1e-3 and info["normAinf"] == 2.25
    assert info["matvecs"] == 48 and info["restarts"] == 2 and info["nullity"] == 1 and info["k0"] == 4


def test_every_corruption_is_an_io_error(ns, tmp_path):
    body = b"NSCKPT01" + record(ns) + bytes(range(200))
    good = write(tmp_path, body, "good.ckpt")
    assert ns.read_checkpoint(good)["k0"] == 4
    cases = {
        "flipped": body[:100] + bytes([body[100] ^ 1]) + body[101:],
        "magic": b"NSCKPT02" + body[8:],
        "version": b"NSCKPT01" + record(ns, version=2) + body[8 + 184:],
    }
    for name, b in cases.items():
        # the flipped body keeps the good body's checksum; the others carry their own
        c = fnv1a_words(body) if name == "flipped" else None
        with pytest.raises(ns.NullspaceError) as e:
            ns.read_checkpoint(write(tmp_path, b, name + ".ckpt", checksum=c))
        assert e.value.status == ns.NS_ERR_IO, name
    raw = good.read_bytes()
    for cut in (0, 7, 8 + 100, len(raw) - 1):
        p = tmp_path / f"cut{cut}.ckpt"
        p.write_bytes(raw[:cut])
        with pytest.raises(ns.NullspaceError) as e:
            ns.read_checkpoint(p)
        assert e.value.status == ns.NS_ERR_IO, cut
    with pytest.raises(ns.NullspaceError) as e:
        ns.read_checkpoint(write(tmp_path, body, "sum.ckpt", checksum=fnv1a_words(body) ^ 1))
    assert e.value.status == ns.NS_ERR_IO
    with pytest.raises(ns.NullspaceError) as e:
        ns.read_checkpoint(tmp_path / "missing.ckpt")
    assert e.value.status == ns.NS_ERR_IO


def test_checksum_is_over_words_not_bytes(ns, tmp_path):
    """The byte-wise FNV-1a of the same body differs; the reader must accept only the
    word-wise one (a check that the format, not some other hash, is implemented)."""
    body = b"NSCKPT01" + record(ns) + b"xyz"
    h = FNV_OFFSET
    for b in body:
        h = ((h ^ b) * FNV_PRIME) & 0xFFFFFFFFFFFFFFFF
    assert h != fnv1a_words(body)
    with pytest.raises(ns.NullspaceError):
        ns.read_checkpoint(write(tmp_path, body, "bytewise.ckpt", checksum=h))
    assert ns.read_checkpoint(write(tmp_path, body, "wordwise.ckpt"))["version"] == 1


def test_checkpoint_options_exist_with_defaults(ns):
    o = ns.default_opts()
    assert o.spmm_schedule == 0 and o.checkpoint_every == 0 and o.resume == 0 and o.checkpoint_path is None
    o = ns.default_opts(checkpoint_path="/tmp/x.ckpt", checkpoint_every=3)
    assert o.checkpoint_path == b"/tmp/x.ckpt" and o.checkpoint_every == 3
