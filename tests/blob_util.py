"""Test helper: serialize an H-matrix given as plain arrays into the version-1
layout documented in include/hmat.h (numpy only; no product code)."""
import struct

import numpy as np

HEADER = 256


def _align(x):
    return (x + 63) // 64 * 64


def write_blob(n, perm, clusters, blocks, block_data, leaf=32, eta=2.0, eps=1e-4):
    """perm[n]; clusters (nc, 4) begin, end, child0, child1; blocks (nb, >=6) i_s, i_e,
    j_s, j_e, kind, rank; block_data[b]: dense (m, n) or (V_m (m, r), W_m (r, n))."""
    perm = np.asarray(perm, dtype=np.int64)
    clusters = np.asarray(clusters, dtype=np.int64)[:, :4]
    blocks = np.asarray(blocks, dtype=np.int64)
    nc, nb = clusters.shape[0], blocks.shape[0]
    flat, offs = [], []
    pos = 0
    dense_e = lr_e = rsum = rmax = 0
    for b in range(nb):
        d = block_data[b]
        if blocks[b, 4] == 0:
            f = np.asarray(d, dtype=np.float64).ravel()
            dense_e += f.size
        else:
            f = np.concatenate([np.asarray(d[0], dtype=np.float64).ravel(), np.asarray(d[1], dtype=np.float64).ravel()])
            lr_e += f.size
            rsum += int(blocks[b, 5])
            rmax = max(rmax, int(blocks[b, 5]))
        offs.append(pos)
        flat.append(f)
        pos += f.size
    data = np.concatenate(flat) if flat else np.zeros(0)
    off_perm = HEADER
    off_cl = _align(off_perm + 8 * n)
    off_bl = _align(off_cl + 32 * nc)
    off_data = _align(off_bl + 64 * nb)
    total = _align(off_data + 8 * data.size)
    buf = np.zeros(total, dtype=np.uint8)
    hdr = b"HMATBLB1" + struct.pack("<II", 1, HEADER)
    hdr += struct.pack("<5q", n, nc, nb, data.size, leaf)
    hdr += struct.pack("<2d", eta, eps)
    hdr += struct.pack("<5q", off_perm, off_cl, off_bl, off_data, total)
    hdr += struct.pack("<4q", dense_e, lr_e, rsum, rmax)
    buf[:len(hdr)] = np.frombuffer(hdr, dtype=np.uint8)
    buf[off_perm:off_perm + 8 * n] = np.frombuffer(perm.tobytes(), dtype=np.uint8)
    buf[off_cl:off_cl + 32 * nc] = np.frombuffer(clusters.tobytes(), dtype=np.uint8)
    bt = np.zeros((nb, 8), dtype=np.int64)
    bt[:, :6] = blocks[:, :6]
    bt[:, 6] = offs
    buf[off_bl:off_bl + 64 * nb] = np.frombuffer(bt.tobytes(), dtype=np.uint8)
    buf[off_data:off_data + 8 * data.size] = np.frombuffer(data.tobytes(), dtype=np.uint8)
    return buf


def oracle_blob(H):
    """Blob of the oracle's own H-matrix (oracle.HMatrix)."""
    idx, _ = H.clusters()
    return write_blob(H.n, H.perm, idx, H.blocks, H.all_block_data(), leaf=H.leaf, eta=H.eta, eps=H.eps)


def dense_blob(A):
    """Blob of an arbitrary small dense matrix: one leaf cluster, one dense block."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    return write_blob(n, np.arange(n), [[0, n, -1, -1]], [[0, n, 0, n, 0, 0]], [A], leaf=max(n, 1))


def read_header(blob):
    hdr = bytes(blob[:HEADER])
    n, nc, nb, nd, leaf = struct.unpack_from("<5q", hdr, 16)
    eta, eps = struct.unpack_from("<2d", hdr, 56)
    off_perm, off_cl, off_bl, off_data, total = struct.unpack_from("<5q", hdr, 72)
    return dict(n=n, nc=nc, nb=nb, nd=nd, leaf=leaf, eta=eta, eps=eps, off_perm=off_perm, off_cl=off_cl,
                off_bl=off_bl, off_data=off_data, total=total)


def read_blob(blob):
    h = read_header(blob)
    b = np.asarray(blob, dtype=np.uint8)
    perm = np.frombuffer(b[h["off_perm"]:h["off_perm"] + 8 * h["n"]].tobytes(), dtype=np.int64)
    cl = np.frombuffer(b[h["off_cl"]:h["off_cl"] + 32 * h["nc"]].tobytes(), dtype=np.int64).reshape(-1, 4)
    bl = np.frombuffer(b[h["off_bl"]:h["off_bl"] + 64 * h["nb"]].tobytes(), dtype=np.int64).reshape(-1, 8)
    data = np.frombuffer(b[h["off_data"]:h["off_data"] + 8 * h["nd"]].tobytes(), dtype=np.float64)
    return h, perm, cl, bl, data
