"""Index arithmetic of the lower-triangle passes (bounds, input layer, output), replayed
on the CPU: the FP32-root decoding of a tile index into (ti, tj), and which elements each
pass writes.  A warp w of a 256-thread block owns rows w, w + 8, ..., w + 56 of a 64 x 64
tile and lane l the columns 2l, 2l + 1; a tile below the diagonal is written directly
and, transposed, to its mirror; a diagonal tile is completed from its lower half."""
import numpy as np

AT = 64


def lower_tile(k):
    """(ti, tj) of lower tile k, tj <= ti, row-major: an FP32 root corrected to the integer."""
    t = int((np.sqrt(np.float32(8.0) * np.float32(k) + np.float32(1.0)) - np.float32(1.0)) * np.float32(0.5))
    while (t + 1) * (t + 2) // 2 <= k:
        t += 1
    while t * (t + 1) // 2 > k:
        t -= 1
    return t, k - t * (t + 1) // 2


def test_lower_tile_inverts_the_row_major_count():
    for nt in (1, 2, 3, 5, 64, 128, 1024):   # n up to 65536
        ks = range(nt * (nt + 1) // 2) if nt <= 128 else list(range(0, 600)) + list(range(523000, 524800))
        for k in ks:
            ti, tj = lower_tile(k)
            assert 0 <= tj <= ti < nt and ti * (ti + 1) // 2 + tj == k


def thread_elements():
    """(r, c) of the 16 elements each of the 256 threads owns in a tile."""
    out = []
    for t in range(256):
        w, lane = t >> 5, t & 31
        out.append([(w + 8 * q, 2 * lane + e) for q in range(8) for e in range(2)])
    return out


def output_writes(n):
    """Count of writes to each D element by the output kernel's tile walk."""
    nt = (n + AT - 1) // AT
    cnt = np.zeros((n, n), int)
    own = thread_elements()
    for k in range(nt * (nt + 1) // 2):
        ti, tj = lower_tile(k)
        i0, j0, dg = ti * AT, tj * AT, ti == tj
        for elems in own:
            for r, c in elems:
                if dg:
                    i, j = i0 + r, i0 + c   # the whole diagonal tile from shared memory
                    if i < n and j < n:
                        cnt[i, j] += 1
                else:
                    if i0 + r < n and j0 + c < n:
                        cnt[i0 + r, j0 + c] += 1     # direct
                    if j0 + r < n and i0 + c < n:
                        cnt[j0 + r, i0 + c] += 1     # mirror
    return cnt


def test_output_writes_every_element_once():
    for n in (1, 63, 64, 65, 130, 301):
        assert np.all(output_writes(n) == 1), n


def test_input_layer_operand_writes_cover_the_padded_matrix_once():
    for np_ in (128, 256):
        nt = np_ // AT
        cnt = np.zeros((np_, np_), int)
        master = np.zeros((np_, np_), int)
        own = thread_elements()
        for k in range(nt * (nt + 1) // 2):
            ti, tj = lower_tile(k)
            i0, j0, dg = ti * AT, tj * AT, ti == tj
            for elems in own:
                for r, c in elems:
                    master[i0 + r, j0 + c] += 1
                    if dg:
                        cnt[i0 + r, i0 + c] += 1
                    else:
                        cnt[i0 + r, j0 + c] += 1
                        cnt[j0 + r, i0 + c] += 1
        assert np.all(cnt == 1)
        low = np.tril(np.ones((np_, np_), bool))
        assert np.all(master[low] == 1)   # the master on and below the diagonal, once


def test_bounds_partials_cover_every_row_and_block_once():
    for n in (1, 64, 65, 200):
        nt = (n + AT - 1) // AT
        cnt = np.zeros((nt, n), int)
        for k in range(nt * (nt + 1) // 2):
            ti, tj = lower_tile(k)
            for t in range(AT):
                if ti * AT + t < n:
                    cnt[tj, ti * AT + t] += 1              # row partials of tile row ti
                if ti != tj and tj * AT + t < n:
                    cnt[ti, tj * AT + t] += 1              # column partials: rows of tile row tj
        assert np.all(cnt == 1), n
