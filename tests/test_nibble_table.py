"""The nibble -> E4M3 table the CUDA decode uses (byte-permute lookup in
csrc/nibble.cuh), checked on the CPU against the E4M3 format's definition
(1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits) for every nibble
and every 16-bit pattern of four nibbles.  The table's constants are read from
the header as text; nothing of the CUDA code runs here."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1503_06202_gb300", "csrc", "nibble.cuh")


def e4m3_code(v: int) -> int:
    """E4M3 bit pattern of a small integer (exact for |v| <= 15)."""
    if v == 0:
        return 0x00
    sign = 0x80 if v < 0 else 0x00
    a = abs(v)
    e = a.bit_length() - 1          # a = 2^e * (1 + m/8)
    mant = (a - (1 << e)) * 8 // (1 << e)
    assert (1 << e) * (8 + mant) == 8 * a, "not exact in E4M3"
    return sign | ((e + 7) << 3) | mant


def prmt(a: int, b: int, s: int, sign_mode: bool) -> int:
    """PTX prmt.b32 default mode (sign_mode) or the CUDA __byte_perm intrinsic
    (selector nibbles taken as 3-bit indices)."""
    pool = [(a >> (8 * i)) & 0xFF for i in range(4)] + [(b >> (8 * i)) & 0xFF for i in range(4)]
    r = 0
    for i in range(4):
        n = (s >> (4 * i)) & 0xF
        byte = pool[n & 7]
        if sign_mode and n & 8:
            byte = 0xFF if byte & 0x80 else 0x00
        r |= byte << (8 * i)
    return r


def table_constants():
    src = open(HEADER).read()
    body = src[src.index("nib4_to_e4m3(uint32_t x)"):]
    body = body[:body.index("}")]
    pos = re.search(r"pos = __byte_perm\((0x[0-9A-Fa-f]+)u, (0x[0-9A-Fa-f]+)u, sel\)", body)
    neg = re.search(r"neg = __byte_perm\((0x[0-9A-Fa-f]+)u, (0x[0-9A-Fa-f]+)u, sel\)", body)
    msk = re.search(r'"r"\((0x[0-9A-Fa-f]+)u\), "r"\(x\)', body)
    assert pos and neg and msk, "table constants not found in nibble.cuh"
    return (int(pos.group(1), 16), int(pos.group(2), 16)), (int(neg.group(1), 16), int(neg.group(2), 16)), \
        int(msk.group(1), 16)


def nib4_to_e4m3(x, pos, neg, msk):
    sel = x & 0x7777
    p = prmt(pos[0], pos[1], sel, False)
    n = prmt(neg[0], neg[1], sel, False)
    m = prmt(msk, msk, x, True)
    return ((p & ~m) | (n & m) | ((m << 1) & 0x80808080)) & 0xFFFFFFFF


def test_e4m3_reference_values():
    # spot values of the format itself (independent of the table)
    assert [e4m3_code(v) for v in (1, 2, 3, 7, -8)] == [0x38, 0x40, 0x44, 0x4E, 0xD0]


def test_nibble_table_matches_e4m3_for_all_patterns():
    pos, neg, msk = table_constants()
    want = [e4m3_code(u - 8) for u in range(16)]
    for x in range(1 << 16):
        got = nib4_to_e4m3(x, pos, neg, msk)
        for i in range(4):
            u = (x >> (4 * i)) & 0xF
            assert (got >> (8 * i)) & 0xFF == want[u], (hex(x), i, u)
