"""Reading and writing grid files byte by byte, for tests that corrupt them.

The file is the header {magic "VDBCGRD1", version, info bytes, activation
bytes, block bytes, table offsets[16], checksum}, then the vdbc_grid_info
struct, the activation flags and the linear block; the checksum is 64-bit
FNV-1a over info, flags and block.  These helpers restate that format from
include/vdbc.h's description so that a test can write a file whose checksum
is right and whose contents are not.
"""
import struct

import numpy as np

HEADER = struct.Struct("<8sIIQQ16QQ")
TILE = 0x80000000
NEURAL = 0x40000000


def fnv1a64(h, data):
    """FNV-1a, 64 bit (Fowler-Noll-Vo)."""
    for byte in data:
        h = ((h ^ byte) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


def read_grid_file(path):
    b = open(path, "rb").read()
    h = HEADER.unpack_from(b, 0)
    info_bytes, active_bytes, block_bytes = h[2], h[3], h[4]
    o = HEADER.size
    assert len(b) == o + info_bytes + active_bytes + block_bytes
    return dict(magic=h[0], version=h[1], offsets=list(h[5:21]), checksum=h[21],
                info=bytearray(b[o:o + info_bytes]),
                active=bytes(b[o + info_bytes:o + info_bytes + active_bytes]),
                block=bytearray(b[o + info_bytes + active_bytes:]))


def write_grid_file(path, f):
    """Writes f with the checksum of its contents."""
    c = fnv1a64(0xCBF29CE484222325, f["info"])
    c = fnv1a64(c, f["active"])
    c = fnv1a64(c, f["block"])
    hdr = HEADER.pack(f["magic"], f["version"], len(f["info"]), len(f["active"]), len(f["block"]),
                      *f["offsets"], c)
    with open(path, "wb") as fh:
        fh.write(hdr + bytes(f["info"]) + bytes(f["active"]) + bytes(f["block"]))


def table(f, k, n):
    """Table k of the block (0 root, 1 upper, 2 lower) as a writable u32 view of n entries."""
    return np.frombuffer(f["block"], dtype=np.uint32, count=n, offset=f["offsets"][k])
