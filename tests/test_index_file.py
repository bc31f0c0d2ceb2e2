"""Index files (pg_index_save / pg_index_load): the host-side checks, run on
CPU through pg_index_file_check against files this test writes from the
layout that include/pg.h documents.  A valid file is accepted; each kind of
damage (checksum, truncation, trailing bytes, foreign magic, version or byte
order, an out-of-range or non-member neighbour, a degree above R, upper
layers that are not ascending subsets of the layer below, a top entry point
outside the top layer) is refused with the documented status, and so is
every one of 2,000 random corruptions."""
import struct

import numpy as np
import pytest

import paper_2410_01231_gb300 as pg

IO, INVALID = 9, 1


def fnv_words(buf: bytes) -> int:
    """FNV-1a over little-endian 64-bit words, the last one zero-padded."""
    h = 0xCBF29CE484222325
    pad = (-len(buf)) % 8
    data = buf + b"\0" * pad
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def tiny_index(n=12, d=8, R=4, M=3, seed=5):
    """A small valid two-layer index: layer 0 a ring graph, layer 1 on the
    even ids with each member linked to the next member."""
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, 256, size=(n, d)).astype(np.float32)
    deg0 = np.full(n, 2, np.int32)
    nbr0 = np.full((n, R), -1, np.int32)
    for u in range(n):
        nbr0[u, 0], nbr0[u, 1] = (u + 1) % n, (u - 1) % n
    gid1 = np.arange(0, n, 2, dtype=np.int32)
    m1 = len(gid1)
    deg1 = np.ones(m1, np.int32)
    nbr1 = np.full((m1, M), -1, np.int32)
    for t in range(m1):
        nbr1[t, 0] = gid1[(t + 1) % m1]
    return dict(n=n, d=d, R=R, M=M, ep_top=0, ep_base=3, pts=pts,
                layers=[(None, deg0, nbr0), (gid1, deg1, nbr1)])


def encode(ix, *, magic=b"PGINDEX\0", version=1, bom=0x01020304, counts=None,
           checksum_delta=0, trailing=b""):
    n, d = ix["n"], ix["d"]
    head = bytearray()
    head += magic + struct.pack("<II", version, bom)
    head += struct.pack("<qiiqq", n, d, 0, ix["ep_top"], ix["ep_base"])
    # metric, precision, K, L, R, M; alpha, alpha_final; iters, connect, route, 0; seed
    head += struct.pack("<iiiiii", 0, 0, 8, 16, ix["R"], ix["M"])
    head += struct.pack("<dd", 66.0, 60.0)
    head += struct.pack("<iiiiQ", 2, 1, 1, 0, 0)
    layers = ix["layers"]
    head += struct.pack("<ii", len(layers), 0)
    for i, (gid, deg, nbr) in enumerate(layers):
        cnt = counts[i] if counts else len(deg)
        head += struct.pack("<qii", cnt, nbr.shape[1], 0 if gid is None else 1)
    body = bytearray(head)
    for gid, deg, nbr in layers:
        if gid is not None:
            body += np.ascontiguousarray(gid, "<i4").tobytes()
        body += np.ascontiguousarray(deg, "<i4").tobytes()
        body += np.ascontiguousarray(nbr, "<i4").tobytes()
    body += np.ascontiguousarray(ix["pts"], "<f4").tobytes()
    s = (fnv_words(bytes(body)) + checksum_delta) & 0xFFFFFFFFFFFFFFFF
    return bytes(body) + struct.pack("<Q", s) + trailing


def check(tmp_path, blob):
    p = tmp_path / "ix.pgi"
    p.write_bytes(blob)
    return pg.index_file_check(str(p))


def refused(tmp_path, blob, status, word):
    with pytest.raises(pg.PGError) as e:
        check(tmp_path, blob)
    assert e.value.status == status, str(e.value)
    assert word in str(e.value), str(e.value)


def test_fnv_words_on_known_inputs():
    # one zero word: offset basis times the prime
    assert fnv_words(b"") == 0xCBF29CE484222325
    assert fnv_words(b"\0" * 8) == (0xCBF29CE484222325 * 0x100000001B3) & (2**64 - 1)
    # a partial word hashes like its zero-padded form
    assert fnv_words(b"\x01") == fnv_words(b"\x01" + b"\0" * 7)


def test_valid_file_is_accepted(tmp_path):
    info = check(tmp_path, encode(tiny_index()))
    assert info == dict(n=12, d=8, n_layers=2)


def test_damaged_points_fail_the_checksum(tmp_path):
    blob = bytearray(encode(tiny_index()))
    blob[-12] ^= 0x40  # inside the last point
    refused(tmp_path, bytes(blob), INVALID, "checksum")
    refused(tmp_path, encode(tiny_index(), checksum_delta=1), INVALID, "checksum")


def test_truncated_and_padded_files(tmp_path):
    blob = encode(tiny_index())
    refused(tmp_path, blob[:-5], IO, "header implies")
    refused(tmp_path, blob[:40], IO, "short read")
    refused(tmp_path, encode(tiny_index(), trailing=b"x"), INVALID, "header implies")


def test_foreign_files(tmp_path):
    refused(tmp_path, encode(tiny_index(), magic=b"NOTANIDX"), INVALID, "not an index file")
    refused(tmp_path, encode(tiny_index(), version=2), INVALID, "version")
    refused(tmp_path, encode(tiny_index(), bom=0x04030201), INVALID, "byte order")
    with pytest.raises(pg.PGError) as e:
        pg.index_file_check(str(tmp_path / "missing.pgi"))
    assert e.value.status == IO


def test_neighbour_out_of_range(tmp_path):
    ix = tiny_index()
    ix["layers"][0][2][5, 1] = ix["n"]
    refused(tmp_path, encode(ix), INVALID, "not a member")
    ix = tiny_index()
    ix["layers"][0][2][5, 0] = -1  # a hole inside the degree
    refused(tmp_path, encode(ix), INVALID, "not a member")


def test_slots_beyond_the_degree_are_not_read(tmp_path):
    ix = tiny_index()
    ix["layers"][0][2][5, 3] = 10**6
    assert check(tmp_path, encode(ix))["n"] == 12


def test_upper_layer_neighbour_must_be_a_member(tmp_path):
    ix = tiny_index()
    ix["layers"][1][2][0, 0] = 1  # odd ids are not in layer 1
    refused(tmp_path, encode(ix), INVALID, "not a member")


def test_degree_above_bound(tmp_path):
    ix = tiny_index()
    ix["layers"][0][1][2] = ix["R"] + 1
    refused(tmp_path, encode(ix), INVALID, "degree")
    ix = tiny_index()
    ix["layers"][1][1][0] = -1
    refused(tmp_path, encode(ix), INVALID, "degree")


def test_upper_layer_members(tmp_path):
    ix = tiny_index()
    g = ix["layers"][1][0]
    g[1], g[2] = g[2], g[1]
    refused(tmp_path, encode(ix), INVALID, "ascending")
    # a third layer with a member missing from layer 1
    ix = tiny_index()
    gid2 = np.array([0, 3], np.int32)
    ix["layers"].append((gid2, np.zeros(2, np.int32), np.full((2, ix["M"]), -1, np.int32)))
    refused(tmp_path, encode(ix), INVALID, "missing from the layer below")


def test_entry_points(tmp_path):
    ix = tiny_index()
    ix["ep_top"] = 1  # not in the top layer (even ids)
    refused(tmp_path, encode(ix), INVALID, "top entry point")
    ix = tiny_index()
    ix["ep_base"] = ix["n"]
    refused(tmp_path, encode(ix), INVALID, "entry point")


def test_layer_shapes(tmp_path):
    ix = tiny_index()
    refused(tmp_path, encode(ix, counts=[11, 6]), INVALID, "shape of layer 0")
    refused(tmp_path, encode(ix, counts=[12, 13]), INVALID, "shape of layer 1")


def test_random_damage_is_always_refused(tmp_path):
    """2,000 random corruptions of a valid file (bit flips, byte runs,
    truncation, extension, spliced headers): each is refused with a status,
    never accepted and never a crash or a huge allocation (the size check
    comes before any array is read)."""
    good = encode(tiny_index())
    rs = np.random.default_rng(77)
    p = tmp_path / "fz.pgi"
    for i in range(2000):
        b = bytearray(good)
        kind = i % 5
        if kind == 0:  # one bit
            j = int(rs.integers(0, len(b)))
            b[j] ^= 1 << int(rs.integers(0, 8))
        elif kind == 1:  # a run of random bytes
            j = int(rs.integers(0, len(b) - 8))
            b[j:j + 8] = rs.integers(0, 256, 8, dtype=np.uint8).tobytes()
        elif kind == 2:  # truncation
            b = b[:int(rs.integers(0, len(b)))]
        elif kind == 3:  # extension
            b += rs.integers(0, 256, int(rs.integers(1, 64)), dtype=np.uint8).tobytes()
        else:  # a huge count or width in the header region
            j = int(rs.integers(16, 200))
            b[j:j + 8] = struct.pack("<q", int(rs.integers(1, 2**62)))
        if bytes(b) == good:
            continue
        p.write_bytes(bytes(b))
        with pytest.raises(pg.PGError) as e:
            pg.index_file_check(str(p))
        assert e.value.status in (IO, INVALID), (i, e.value.status)
