"""Shared-memory pitches of the FFT kernels, restated on the host: the
claims their comments make about 8-byte accesses of a half-warp (16 lanes,
one bank pair per 8-byte slot, 16 bank pairs) hold for every size the
kernels use. seq_pitch (x2 and x3 passes) keeps C sequences 16/C (mod 16)
slots apart; pitch3 (3 x N row kernels) keeps the three decimated buffers
11 (mod 16) slots apart."""


def seq_pitch(n, c):
    pad = ((16 // c) - n) % 16
    return n + (16 if pad == 0 else pad)


def pitch3(n):
    return n + (11 - n) % 16


def bank_pairs(slots):
    return len({s % 16 for s in slots})


def test_seq_pitch_epilogue_reads_hit_sixteen_bank_pairs():
    # lanes of a half-warp: column c = lane % C, element s0 + lane // C
    for n in [2 ** k for k in range(4, 14)] + [3 * 2 ** k for k in range(4, 12)]:
        for c in (2, 4, 8, 16):
            ld = seq_pitch(n, c)
            assert ld > n and ld % 16 == (16 // c) % 16
            for s0 in range(0, n - 16):
                slots = [(lane % c) * ld + s0 + lane // c for lane in range(16)]
                assert bank_pairs(slots) == 16, (n, c, s0)


def test_pitch3_decimated_accesses_hit_sixteen_bank_pairs():
    # sample j of a row lives in buffer j % 3, slot j // 3
    for n in (256, 512):
        lb = pitch3(n)
        assert lb >= n and lb % 16 == 11
        for j0 in range(0, 3 * n - 16):
            slots = [(j % 3) * lb + j // 3 for j in range(j0, j0 + 16)]
            assert bank_pairs(slots) == 16, (n, j0)


def test_unpadded_layouts_conflict():
    # the layouts these pitches replaced: pitch n + 1 for C = 8, and buffers
    # n apart, hit fewer bank pairs
    assert bank_pairs([(lane % 8) * 1025 + lane // 8 for lane in range(16)]) < 16
    assert bank_pairs([(j % 3) * 512 + j // 3 for j in range(16)]) < 16
