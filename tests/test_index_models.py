"""Models of two kernels' work decomposition, run on the CPU.

Each model restates, in numpy and per thread, how a kernel splits its work:
which thread reads which value, where it adds or stores it, and in which
shared-memory slot.  It then checks the result against a plain definition.
The models neither call nor share code with the kernels or the oracle.  They
pin the index arithmetic, and the GPU parity tests pin the kernels.

- k_deposit (Eq. (rhodis), cloud-in-cell): a warp owns a tile of TY x TZ mesh
  rows, takes each plane's source rows as chains of records in batches of 32,
  sums equal cells, then adds f_x and 1 - f_x in separate steps and the two
  destination-row phases one after the other.  The model checks that no two
  lanes of one step add to the same slot, that every slot index and output
  row lies in bounds, and that the result equals the direct deposit.  It runs
  on meshes of 1 to 12 cells (where the periodic images of a tile's rows
  coincide) for every tile shape and several warps per block.
- k_xy_r2c / k_xy_c2r (the x and y transforms of a 256^2 plane): the model
  runs the four-step factorisations, the real-to-complex packing, the
  packed x = 0 / x = N/2 column and the exchange between the eight CTAs of a
  cluster.  It checks the result against numpy's rfft2 and irfft2 (both
  unnormalised).
"""
import itertools

import numpy as np


# ---------------------------------------------------------------- deposit
def _wrap(i, n):
    return i + n if i < 0 else (i - n if i >= n else i)


def _deposit_model(cells, f, n, TY, TZ, nw):
    order = np.argsort(cells, kind="stable")
    cells, f = cells[order], f[order]
    npart = len(cells)
    row_start = np.searchsorted(cells // n, np.arange(n * n + 1), side="left")
    q = 4
    stride = (n + 1 + q - 1) // q * q
    rho = np.full(n ** 3, np.nan)
    written = np.zeros(n ** 3, int)
    span_y = nw * TY
    tiles_y = (n + span_y - 1) // span_y
    for blk in range(tiles_y * ((n + TZ - 1) // TZ)):
        for warp in range(nw):
            y0, z0 = (blk % tiles_y) * span_y + warp * TY, (blk // tiles_y) * TZ
            if y0 >= n:
                continue
            ty, tz = min(TY, n - y0), min(TZ, n - z0)
            acc = np.zeros(TY * TZ * stride)
            nr = (tz + 1) * (ty + 1)
            lanes = range(nr)
            sz_l = [L // (ty + 1) for L in range(32)]
            ly_l = [L - sz_l[L] * (ty + 1) for L in range(32)]
            b, e, base, head = [0] * 32, [0] * 32, [0] * 32, [False] * 32
            for L in lanes:
                yr = _wrap(y0 - 1 + ly_l[L], n)
                srow = _wrap(z0 - 1 + sz_l[L], n) * n + yr
                b[L], e[L], base[L] = row_start[srow], min(row_start[srow + 1], npart), srow * n
                head[L] = ly_l[L] == 0 or yr != _wrap(y0 - 2 + ly_l[L], n) + 1
            heads = [L for L in range(32) if head[L]]
            last = [((min([h for h in heads if h > L], default=nr)) - 1) for L in range(32)]
            for k in [L for L in range(32) if head[L] and b[L] < e[max(last[L], 0)]]:
                j, en, nrc = b[k], e[last[k]], last[k] - k + 1
                while j < en:
                    idx = range(j, min(j + 32, en))
                    lanes_b = []
                    for t, i in enumerate(idx):
                        rel = (int(cells[i]) - base[k]) % 2 ** 32
                        off = rel // n
                        ok = off < nrc
                        fx, fy, fz = f[i]
                        v = np.zeros((2, 2, 2))
                        for dz, dy in itertools.product((0, 1), repeat=2):
                            w = (fy if dy else 1 - fy) * (fz if dz else 1 - fz)
                            v[dy, dz, 1], v[dy, dz, 0] = fx * w, (1 - fx) * w
                        lanes_b.append((rel if ok else 0x80000000 + t, ok, ly_l[k] + off, rel - off * n, v))
                    adds, t = [], 0
                    while t < len(lanes_b):  # runs of equal cells: the run's last lane adds the sum
                        u, tot = t, lanes_b[t][4].copy()
                        while u + 1 < len(lanes_b) and lanes_b[u + 1][0] == lanes_b[t][0]:
                            u += 1
                            tot += lanes_b[u][4]
                        if lanes_b[u][1]:
                            adds.append((lanes_b[u][2], lanes_b[u][3], tot))
                        t = u + 1
                    sz = sz_l[k]
                    for dy in (0, 1):
                        for hi in (1, 0):
                            seen = set()
                            for ly, x, tot in adds:
                                ry = ly - 1 + dy
                                for dz in (0, 1):
                                    lz = sz - 1 + dz
                                    if 0 <= ry < ty and 0 <= lz < tz:
                                        a = (lz * TY + ry) * stride + x + hi
                                        assert 0 <= a < TY * TZ * stride
                                        assert a not in seen, "two lanes of one step add to one slot"
                                        seen.add(a)
                                        acc[a] += tot[dy, dz, hi]
                    j += 32
            for lz in range(tz):
                for ry in range(ty):
                    a0 = (lz * TY + ry) * stride
                    acc[a0] += acc[a0 + n]
                    o = ((z0 + lz) * n + y0 + ry) * n
                    assert o + n <= n ** 3
                    rho[o:o + n] = acc[a0:a0 + n]
                    written[o:o + n] += 1
    assert (written == 1).all(), "every output row written exactly once"
    return rho.reshape(n, n, n)


def _direct_deposit(cells, f, n):
    rho = np.zeros((n, n, n))
    for c, (fx, fy, fz) in zip(cells, f):
        z, r = divmod(int(c), n * n)
        y, x = divmod(r, n)
        for dz, dy, dx in itertools.product((0, 1), repeat=3):
            w = (fz if dz else 1 - fz) * (fy if dy else 1 - fy) * (fx if dx else 1 - fx)
            rho[(z + dz) % n, (y + dy) % n, (x + dx) % n] += w
    return rho


def test_deposit_tiles_chains_and_phases_cover_every_node_once():
    rng = np.random.default_rng(1)
    for n in (1, 2, 3, 5, 8, 12):
        for npart, clustered in ((0, False), (3, False), (n ** 3 // 8 + 3, False), (2 * n ** 3, True)):
            side = min(3, n) if clustered else n
            cells = rng.integers(0, side, size=(npart, 3))
            c = ((cells[:, 2] * n + cells[:, 1]) * n + cells[:, 0]).astype(np.uint32)
            f = rng.random((npart, 3))
            ref = _direct_deposit(c, f, n)
            for TY, TZ in ((2, 4), (2, 2), (1, 2), (1, 1)):
                for nw in (1, 3):
                    got = _deposit_model(c, f, n, TY, TZ, nw)
                    np.testing.assert_allclose(got, ref, atol=1e-12, err_msg=str((n, npart, TY, TZ, nw)))


# ---------------------------------------------------------------- x-y transforms of a 256^2 plane
XY_N, XY_CL = 256, 8
XY_ROWS, XY_COLS, XY_SROW = XY_N // XY_CL, XY_N // 2 // XY_CL, 136
W256 = np.exp(-2j * np.pi * np.arange(256) / 256)


def _bitrev(k, m):
    r, b = 0, 1
    while b < m:
        r = (r << 1) | (1 if k & b else 0)
        b <<= 1
    return r


def _dft_bitrev(a, inv):
    """The in-register DFT along the last axis: natural order in, bit-reversed out."""
    m = a.shape[-1]
    s = 1 if inv else -1
    mat = np.exp(s * 2j * np.pi * np.outer(np.arange(m), np.arange(m)) / m)
    x = a @ mat
    out = np.empty_like(x)
    for k in range(m):
        out[..., _bitrev(k, m)] = x[..., k]
    return out


def _sw(n):
    return n + (n >> 4)


def _x_rows_forward(rows):
    """Rows (R, 256) real -> X[k] for k < 128 per row (k = 0 packed), thread by thread: thread j of a
    row holds z[j + 8m]; after the exchange thread j holds Z[k1 + 16 k2], k1 = 2j + h; the partner
    lanes supply Z[128 - k]."""
    R = rows.shape[0]
    z = rows[:, 0::2] + 1j * rows[:, 1::2]  # (R, 128)
    S = np.zeros((R, XY_SROW), complex)
    a = _dft_bitrev(np.stack([z[:, j::8] for j in range(8)], axis=1), False)  # (R, 8 threads, 16)
    for j in range(8):
        for k1 in range(16):
            S[:, _sw(j + 8 * k1)] = a[:, j, _bitrev(k1, 16)] * W256[(2 * j * k1) & 255]
    Z = np.zeros((R, 8, 2, 8), complex)  # [row][lane j][h][k2]
    for j in range(8):
        for h in range(2):
            k1 = 2 * j + h
            b = _dft_bitrev(np.stack([S[:, _sw(jj + 8 * k1)] for jj in range(8)], axis=1), False)
            for k2 in range(8):
                Z[:, j, h, k2] = b[:, _bitrev(k2, 8)]
    X = np.zeros((R, 128), complex)
    for j in range(8):
        for k2 in range(8):
            zp0 = Z[:, 0, 0, (8 - k2) & 7] if j == 0 else Z[:, (8 - j) & 7, 0, 7 - k2]
            zp1 = Z[:, 7 - j, 1, 7 - k2]
            for h, zp in ((0, zp0), (1, zp1)):
                k = 2 * j + h + 16 * k2
                zk = Z[:, j, h, k2]
                E, O = 0.5 * (zk + np.conj(zp)), -0.5j * (zk - np.conj(zp))
                X[:, k] = (E.real + O.real) + 1j * (E.real - O.real) if k == 0 else E + W256[k] * O
    return X


def _xy_forward_model(plane):
    T = [np.zeros(max(XY_N * XY_COLS, XY_ROWS * XY_SROW), complex) for _ in range(XY_CL)]
    for q in range(XY_CL):  # x phase: each CTA's rows, stored row after row
        X = _x_rows_forward(plane[XY_ROWS * q:XY_ROWS * (q + 1)])
        for r in range(XY_ROWS):
            T[q][r * XY_SROW:r * XY_SROW + 128] = X[r]
    spec = np.full((256, 129), np.nan, complex)
    for q in range(XY_CL):  # y phase: CTA q pulls its 16 columns of every row from the rows' owners
        u = np.zeros((XY_COLS, 16, 16), complex)  # [column c][thread jt][mm]
        for c in range(XY_COLS):
            for jt in range(16):
                for mm in range(16):
                    yy = jt + 16 * mm
                    idx = (yy % XY_ROWS) * XY_SROW + XY_COLS * q + c
                    assert 0 <= idx < len(T[0])
                    u[c, jt, mm] = T[yy // XY_ROWS][idx]
        u = _dft_bitrev(u, False)
        Ty = np.zeros((256, XY_COLS), complex)
        for jt in range(16):
            for k1 in range(16):
                Ty[jt + 16 * k1] = u[:, jt, _bitrev(k1, 16)] * W256[(jt * k1) & 255]
        v = _dft_bitrev(np.stack([Ty[16 * jt:16 * jt + 16].T for jt in range(16)], axis=1), False)
        for c in range(XY_COLS):
            kx = XY_COLS * q + c
            col = np.array([v[c, ky % 16, _bitrev(ky // 16, 16)] for ky in range(256)])
            if kx == 0:
                mirror = col[(-np.arange(256)) % 256]
                spec[:, 0] = 0.5 * (col + np.conj(mirror))
                spec[:, 128] = -0.5j * (col - np.conj(mirror))
            else:
                spec[:, kx] = col
    return spec


def _xy_inverse_model(spec):
    T = [np.zeros(max(XY_N * XY_COLS, XY_ROWS * XY_SROW), complex) for _ in range(XY_CL)]
    for q in range(XY_CL):  # y phase: each CTA's columns (kx = 0 packed with kx = N/2)
        cols = []
        for c in range(XY_COLS):
            kx = XY_COLS * q + c
            cols.append(spec[:, 0] + 1j * spec[:, 128] if kx == 0 else spec[:, kx])
        cols = np.array(cols)  # (16, 256)
        u = _dft_bitrev(np.stack([cols[:, jt::16] for jt in range(16)], axis=1), True)
        Ty = np.zeros((256, XY_COLS), complex)
        for jt in range(16):
            for k1 in range(16):
                Ty[jt + 16 * k1] = u[:, jt, _bitrev(k1, 16)] * np.conj(W256[(jt * k1) & 255])
        v = _dft_bitrev(np.stack([Ty[16 * jt:16 * jt + 16].T for jt in range(16)], axis=1), True)
        for jt in range(16):
            for k2 in range(16):
                T[q][(jt + 16 * k2) * XY_COLS:(jt + 16 * k2 + 1) * XY_COLS] = v[:, jt, _bitrev(k2, 16)]
    out = np.full((256, 256), np.nan)
    for q in range(XY_CL):  # x phase: row y's X[k] pulled from column owner k / 16
        R = XY_ROWS
        a = np.zeros((R, 8, 16), complex)
        pulled = np.zeros((R, 8, 16), complex)
        for r in range(R):
            y = XY_ROWS * q + r
            for j in range(8):
                for m in range(16):
                    k = j + 8 * m
                    pulled[r, j, m] = T[k // XY_COLS][y * XY_COLS + (k % XY_COLS)]
        for j in range(8):
            for m in range(16):  # the mirrored value: the partner lane's pull (or this lane's, j = 0)
                k = j + 8 * m
                xk = pulled[:, j, m]
                xp = pulled[:, 0, (16 - m) & 15] if j == 0 else pulled[:, 8 - j, 15 - m]
                if k == 0:
                    a[:, j, m] = (xk.real + xk.imag) + 1j * (xk.real - xk.imag)
                else:
                    e, d = xk + np.conj(xp), np.conj(W256[k]) * (xk - np.conj(xp))
                    a[:, j, m] = e + 1j * d
        a = _dft_bitrev(a, True)
        S = np.zeros((R, XY_SROW), complex)
        for j in range(8):
            for k1 in range(16):
                S[:, _sw(j + 8 * k1)] = a[:, j, _bitrev(k1, 16)] * np.conj(W256[(2 * j * k1) & 255])
        for j in range(8):
            for h in range(2):
                k1 = 2 * j + h
                b = _dft_bitrev(np.stack([S[:, _sw(jj + 8 * k1)] for jj in range(8)], axis=1), True)
                for k2 in range(8):
                    nn = k1 + 16 * k2
                    out[XY_ROWS * q:XY_ROWS * (q + 1), 2 * nn] = b[:, _bitrev(k2, 8)].real
                    out[XY_ROWS * q:XY_ROWS * (q + 1), 2 * nn + 1] = b[:, _bitrev(k2, 8)].imag
    return out


def test_xy_transform_decomposition_matches_rfft2_and_irfft2():
    rng = np.random.default_rng(7)
    plane = rng.standard_normal((256, 256))
    spec = _xy_forward_model(plane)
    ref = np.fft.rfft2(plane)
    assert np.abs(spec - ref).max() < 1e-9 * np.abs(ref).max()
    back = _xy_inverse_model(ref)
    ref_back = np.fft.irfft2(ref, s=(256, 256)) * 256 * 256  # unnormalised, like the C2R
    assert np.abs(back - ref_back).max() < 1e-9 * np.abs(ref_back).max()
