"""Table 1 (Section 3.4) pinned cell by cell on a hand-written H-matrix.

The H-matrix has N = 4 unknowns, one dense block A|^1 (rows 0-1, columns 0-1)
and one rank-2 block V_2 W_2 (rows 0-1, columns 2-3).  Its entries are exact in
FP32 (so rounding the matrix to FP32 loses nothing by itself) and the source
vector carries bits below FP32 resolution, so every precision choice of Table 1
shows in the result bits:

  * a product of two FP32 operands is rounded to FP32 (C/Fortran promotion,
    Section 3.4, last paragraph) -- promoting it instead changes the bits;
  * Method 1 keeps z_m = W_m x_m in FP32 -- keeping it in FP64 changes the bits;
  * Method 1-Mixed rounds z_m after each FP64 update z + w x;
  * Methods 2 and 3 keep z_m in FP64 and scale it by D_m (eq. 23).

Each expected value below is written with numpy float32 / float64 scalar
arithmetic, one statement per cell of Table 1, and compared with the oracle bit
for bit.  A second check makes sure the chosen entries really discriminate: each
plausible misreading (a promoted product, an FP64 z_m, an FP32 source where
Table 1 says FP64) gives different bits.
"""
import os

import numpy as np
import pytest

f32, f64 = np.float32, np.float64
E = 2.0 ** -12
A1 = [[1 + E, 3 * E], [1 - E, 1 + 3 * E]]                 # dense A|^1, 2 x 2
V2 = [[3.0, 2.0 ** -10], [1 + E, -(2.0 ** -11)]]           # V_2, 2 x 2 (rows x ranks)
# W_2, 2 x 2 (ranks x columns), and the FP64 source x.  Rank 1 of Method
# 1-Single: its first term leaves z = w x = 4 + 2^-21 (exact), an odd FP32 value
# (ulp 2^-21); its second product w x = 2^-22 (1 - 2^-28) rounds to exactly 2^-22
# in FP32, so z + fl32(w x) is a tie that rounds up (to even), while z + w x
# taken in FP64 sits just below the tie and rounds down.
W2 = [[4 + 2.0 ** -21, 2.0 ** -22 * (1 + 2.0 ** -14)], [2.0 ** -9, 3 * 2.0 ** -10]]
X = [1 + E + 2.0 ** -40, 1 + 2.0 ** -30, 1 + 2.0 ** -40, 1 - 2.0 ** -14 + 2.0 ** -38]


def _hmat(oracle_mod):
    return oracle_mod.HMatrix.from_blocks(4, [(0, 2, 0, 2, np.array(A1)), (0, 2, 2, 4, (np.array(V2), np.array(W2)))])


def _method2_factors():
    """eq. (11)-(16): V'_l = V_l / max|V_l|, W'_l = W_l / max|W_l|, d_l the product
    of the two maxima (all powers of two or exact quotients here)."""
    Vp = [[0.0, 0.0], [0.0, 0.0]]
    Wp = [[0.0, 0.0], [0.0, 0.0]]
    d = [0.0, 0.0]
    for l in range(2):
        dv = max(abs(V2[0][l]), abs(V2[1][l]))
        dw = max(abs(W2[l][0]), abs(W2[l][1]))
        for i in range(2):
            Vp[i][l] = f64(V2[i][l]) / f64(dv)
        for j in range(2):
            Wp[l][j] = f64(W2[l][j]) / f64(dw)
        d[l] = f64(dv) * f64(dw)
    return Vp, Wp, d


# ---- the dense step (eq. 21), one function per Table 1 row group ----
def dense_fp64(i):                     # y^ FP64, A FP64, x FP64
    y = f64(0)
    for j in range(2):
        y = y + f64(A1[i][j]) * f64(X[j])
    return y


def dense_single(i, promote=False):    # y^ FP64, A FP32, x FP32: FP32 x FP32 -> FP32, then promoted
    y = f64(0)
    for j in range(2):
        p = f64(f32(A1[i][j])) * f64(f32(X[j])) if promote else f64(f32(A1[i][j]) * f32(X[j]))
        y = y + p
    return y


def dense_mixed(i, x32=False):         # y^ FP64, A FP32, x FP64: FP32 A promoted
    y = f64(0)
    for j in range(2):
        xj = f64(f32(X[j])) if x32 else f64(X[j])
        y = y + f64(f32(A1[i][j])) * xj
    return y


# ---- the low-rank step of each method (eq. 9-10, 22-25) ----
def lr_m1_double():
    z = [f64(0), f64(0)]
    for l in range(2):
        for j in range(2):
            z[l] = z[l] + f64(W2[l][j]) * f64(X[2 + j])           # z FP64, W FP64, x FP64
    return [f64(0) + f64(V2[i][0]) * z[0] + f64(V2[i][1]) * z[1] for i in range(2)]


def lr_m1_single(promote_wx=False, promote_vz=False, z64=False):
    z = [f64(0) if z64 else f32(0)] * 2
    for l in range(2):
        for j in range(2):
            w, x = f32(W2[l][j]), f32(X[2 + j])                      # W FP32, x FP32
            if z64:
                z[l] = z[l] + f64(w * x)
            elif promote_wx:
                z[l] = f32(f64(z[l]) + f64(w) * f64(x))
            else:
                z[l] = z[l] + w * x                                  # FP32 x FP32 -> FP32, z FP32
    out = []
    for i in range(2):
        y = f64(0)                                                   # y^ FP64
        for l in range(2):
            v = f32(V2[i][l])                                        # V FP32
            y = y + (f64(v) * f64(z[l]) if (promote_vz or z64) else f64(v * z[l]))
        out.append(y)
    return out


def lr_m1_mixed(z64=False, promote=False):
    z = [f64(0) if z64 else f32(0)] * 2
    for l in range(2):
        for j in range(2):
            t = f64(z[l]) + f64(f32(W2[l][j])) * f64(X[2 + j])      # W FP32 promoted, x FP64
            z[l] = t if z64 else f32(t)                              # z FP32: each update rounded
    out = []
    for i in range(2):
        y = f64(0)
        for l in range(2):
            v = f32(V2[i][l])
            y = y + (f64(v) * f64(z[l]) if (promote or z64) else f64(v * f32(z[l])))  # FP32 x FP32
        out.append(y)
    return out


def lr_m2(kind, rank64=(False, False), promote=False, z32=False, x32=False):
    """Method 2 (and Method 3 via rank64: the ranks kept FP64 run as Method
    2-Double, the others as `kind`; the two partial y^ are added, Section 3.4)."""
    Vp, Wp, d = _method2_factors()
    y64, y32 = [f64(0), f64(0)], [f64(0), f64(0)]
    for l in range(2):
        z = f64(0)                                                   # z FP64 (Table 1, Method 2)
        for j in range(2):
            if rank64[l] or kind == "double":
                z = z + f64(Wp[l][j]) * f64(X[2 + j])                # W' FP64, x FP64
            elif kind == "single":
                w, x = f32(Wp[l][j]), f32(X[2 + j])                  # W' FP32, x FP32
                z = z + (f64(w) * f64(x) if promote else f64(w * x))
            else:
                x = f64(f32(X[2 + j])) if x32 else f64(X[2 + j])     # W' FP32 promoted, x FP64
                z = z + f64(f32(Wp[l][j])) * x
            if z32:
                z = f64(f32(z))
        z = z * d[l]                                                 # D FP64 (eq. 23)
        for i in range(2):
            if rank64[l] or kind == "double":
                y64[i] = y64[i] + f64(Vp[i][l]) * z                  # V' FP64
            else:
                y32[i] = y32[i] + f64(f32(Vp[i][l])) * z             # V' FP32 promoted, z FP64
    return [y64[i] + y32[i] for i in range(2)]


def assemble(dense, lr):
    """eq. (25): the blocks' y^ added into y in block order (rows 2-3 have no block)."""
    return np.array([(f64(0) + dense[i]) + lr[i] for i in range(2)] + [0.0, 0.0])


def expected(name):
    if name == "M1_DOUBLE":
        return assemble([dense_fp64(i) for i in range(2)], lr_m1_double())
    if name == "M1_SINGLE":
        return assemble([dense_single(i) for i in range(2)], lr_m1_single())
    if name == "M1_MIXED":
        return assemble([dense_mixed(i) for i in range(2)], lr_m1_mixed())
    if name == "M2_DOUBLE":
        return assemble([dense_fp64(i) for i in range(2)], lr_m2("double"))
    if name == "M2_SINGLE":
        return assemble([dense_single(i) for i in range(2)], lr_m2("single"))
    if name == "M2_MIXED":
        return assemble([dense_mixed(i) for i in range(2)], lr_m2("mixed"))
    raise KeyError(name)


# the misreadings that must show in the bits
MISREADINGS = {
    "M1_SINGLE": {
        "dense FP32 products promoted": lambda: assemble([dense_single(i, promote=True) for i in range(2)], lr_m1_single()),
        "W x products promoted": lambda: assemble([dense_single(i) for i in range(2)], lr_m1_single(promote_wx=True)),
        "V z products promoted": lambda: assemble([dense_single(i) for i in range(2)], lr_m1_single(promote_vz=True)),
        "z_m kept in FP64": lambda: assemble([dense_single(i) for i in range(2)], lr_m1_single(z64=True)),
    },
    "M1_MIXED": {
        "z_m kept in FP64": lambda: assemble([dense_mixed(i) for i in range(2)], lr_m1_mixed(z64=True)),
        "V z product promoted": lambda: assemble([dense_mixed(i) for i in range(2)], lr_m1_mixed(promote=True)),
        "FP32 source in the dense step": lambda: assemble([dense_mixed(i, x32=True) for i in range(2)], lr_m1_mixed()),
    },
    "M2_SINGLE": {
        "dense FP32 products promoted": lambda: assemble([dense_single(i, promote=True) for i in range(2)], lr_m2("single")),
        "W' x products promoted": lambda: assemble([dense_single(i) for i in range(2)], lr_m2("single", promote=True)),
        "z_m rounded to FP32": lambda: assemble([dense_single(i) for i in range(2)], lr_m2("single", z32=True)),
    },
    "M2_MIXED": {
        "z_m rounded to FP32": lambda: assemble([dense_mixed(i) for i in range(2)], lr_m2("mixed", z32=True)),
        "FP32 source in the low-rank step": lambda: assemble([dense_mixed(i) for i in range(2)], lr_m2("mixed", x32=True)),
    },
}

# the cells each expected value above implements, in the golden file's column order:
# dense:yhat dense:A dense:x lr:z lr:W' lr:x lr:D lr:yhat lr:V' result:y
CELLS = {
    "M1_DOUBLE": "FP64 FP64 FP64 FP64 FP64 FP64 - FP64 FP64 FP64",
    "M1_SINGLE": "FP64 FP32 FP32 FP32 FP32 FP32 - FP64 FP32 FP64",
    "M1_MIXED": "FP64 FP32 FP64 FP32 FP32 FP64 - FP64 FP32 FP64",
    "M2_DOUBLE": "FP64 FP64 FP64 FP64 FP64 FP64 FP64 FP64 FP64 FP64",
    "M2_SINGLE": "FP64 FP32 FP32 FP64 FP32 FP32 FP64 FP64 FP32 FP64",
    "M2_MIXED": "FP64 FP32 FP64 FP64 FP32 FP64 FP64 FP64 FP32 FP64",
}


def _golden():
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "table1_precision.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = f[1:]
    return rows


def test_entries_are_fp32_exact_and_source_is_not():
    for v in [a for r in A1 for a in r] + [a for r in V2 for a in r] + [a for r in W2 for a in r]:
        assert f64(f32(v)) == v
    assert all(f64(f32(x)) != x for x in X)


@pytest.mark.parametrize("name", list(CELLS))
def test_cells_match_the_golden_table(name):
    assert _golden()[name] == CELLS[name].split()


@pytest.mark.parametrize("name", list(CELLS))
def test_oracle_matches_table1_cell_by_cell(oracle_mod, name):
    H = _hmat(oracle_mod)
    y = H.matvec(np.array(X), oracle_mod.VARIANTS[name])
    assert np.array_equal(y, expected(name)), (y, expected(name))


@pytest.mark.parametrize("name", list(MISREADINGS))
def test_each_misreading_changes_the_bits(name):
    good = expected(name)
    for what, alt in MISREADINGS[name].items():
        assert not np.array_equal(alt(), good), f"{name}: '{what}' is not visible with these entries"


@pytest.mark.parametrize("c,rank64", [(-1, (False, False)), (1, (True, False)), (6, (True, False)), (7, (True, True))])
def test_method3_split_cell_by_cell(oracle_mod, c, rank64):
    """Method 3 (eq. 17-20): rank l is FP64 iff d_l >= d_max 10^-c; here d_2 / d_1 is
    about 3.7e-7, so c = 1..6 demotes rank 2 only and c = 7 keeps both (c = -1
    demotes both).  The dense block stays FP64; the FP64 ranks run as Method
    2-Double and the FP32 ranks as Method 2-Mixed, the two y^ added."""
    _, _, d = _method2_factors()
    assert [d[l] >= max(d) * 10.0 ** (-c) for l in range(2)] == list(rank64)
    H = _hmat(oracle_mod)
    y = H.matvec(np.array(X), oracle_mod.M3, c=c)
    want = assemble([dense_fp64(i) for i in range(2)], lr_m2("mixed", rank64=rank64))
    assert np.array_equal(y, want), (y, want)
