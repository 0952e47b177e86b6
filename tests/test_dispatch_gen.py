"""The generated shifted-add dispatch of the dedispersion kernel (A5,
Sec. 2.2.2), checked symbolically on the CPU: for every block of every
generated function, each accumulator receives exactly the staged samples the
definition D[d][t] = sum_c y[c][t + delay[d][c]] asks of it, each once.

The blocks are parsed from the generator's inline-assembly text; a window
register stands for the staged sample (or half-word, or word) it was loaded
from, so a wrong offset, a missing or a doubled add, or a pair formed from the
wrong samples fails here without a GPU."""
import os
import re
import sys
from collections import defaultdict

import pytest

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", "paper_1307_5700_gb300", "csrc"))
import gen_dispatch as G  # noqa: E402


def _blocks(text):
    """{block index: [instruction, ...]} from a generated function."""
    out, cur = {}, None
    for raw in text.splitlines():
        m = re.match(r'\s*"(.*)\\n"\s*$', raw)
        if not m:
            continue
        ins = m.group(1).strip()
        lab = re.fullmatch(r"C(\d+):", ins)
        if lab:
            cur = int(lab.group(1))
            out[cur] = []
        elif ins == "CEND:":
            cur = None
        elif cur is not None and not ins.startswith("bra.uni"):
            out[cur].append(ins)
    return out


def _load_offsets(ins):
    m = re.fullmatch(r"ld\.shared\.(?:f32|b32) (\w+), \[%\d+\+(\d+)\];", ins)
    return (m.group(1), int(m.group(2))) if m else None


@pytest.mark.parametrize("S,MMAX", G.QUADS)
def test_quads_fp32(S, MMAX):
    for b, body in _blocks(G.emit_quad(S, MMAX)).items():
        o = G.quad_steps(b)
        reg, acc = {}, defaultdict(list)
        for ins in body:
            ld = _load_offsets(ins)
            if ld:
                reg[ld[0]] = ld[1] // 4
                continue
            m = re.fullmatch(r"add\.f32 %(\d+), %\1, (\w+);", ins)
            assert m, ins
            acc[int(m.group(1))].append(reg[m.group(2)])
        for j in range(4):
            for s in range(S):
                assert acc[j * S + s] == [s + o[j]], (b, j, s)
        assert len(acc) == 4 * S


@pytest.mark.parametrize("S,MMAX", G.QUADS2)
def test_quads_two_segments(S, MMAX):
    for b, body in _blocks(G.emit_quad2(S, MMAX)).items():
        o = G.quad_steps(b)
        reg, pair, lo, hi = {}, {}, defaultdict(list), defaultdict(list)
        for ins in body:
            ld = _load_offsets(ins)
            if ld:
                off = ld[1] // 4
                # segment 1's window starts 32 S samples after segment 0's
                reg[ld[0]] = (1, off - 32 * S) if off >= 32 * S else (0, off)
                continue
            m = re.fullmatch(r"mov\.b64 (\w+), \{(\w+), (\w+)\};", ins)
            if m:
                pair[m.group(1)] = (reg[m.group(2)], reg[m.group(3)])
                continue
            m = re.fullmatch(r"add\.rn\.f32x2 %(\d+), %\1, (\w+);", ins)
            assert m, ins
            r = int(m.group(1))
            lo[r].append(pair[m.group(2)][0])
            hi[r].append(pair[m.group(2)][1])
        for j in range(4):
            for s in range(S):
                assert lo[j * S + s] == [(0, s + o[j])], (b, j, s)
                assert hi[j * S + s] == [(1, s + o[j])], (b, j, s)


@pytest.mark.parametrize("S,MMAX", G.QUADSP)
def test_quads_in_lane_pairs(S, MMAX):
    H = S // 2
    for b, body in _blocks(G.emit_quadp(S, MMAX)).items():
        o = G.quad_steps(b)
        reg, pair = {}, {}
        lo, hi, tail = defaultdict(list), defaultdict(list), defaultdict(list)
        for ins in body:
            ld = _load_offsets(ins)
            if ld:
                reg[ld[0]] = ld[1] // 4
                continue
            m = re.fullmatch(r"mov\.b64 (\w+), \{(\w+), (\w+)\};", ins)
            if m:
                pair[m.group(1)] = (reg[m.group(2)], reg[m.group(3)])
                continue
            m = re.fullmatch(r"add\.rn\.f32x2 %(\d+), %\1, (\w+);", ins)
            if m:
                r = int(m.group(1))
                lo[r].append(pair[m.group(2)][0])
                hi[r].append(pair[m.group(2)][1])
                continue
            m = re.fullmatch(r"add\.rn\.f32 %(\d+), %\1, (\w+);", ins)
            assert m, ins
            tail[int(m.group(1))].append(reg[m.group(2)])
        for j in range(4):
            for s in range(H):
                # outputs s (low word) and s + H (high word) of trial j
                assert lo[j * H + s] == [s + o[j]], (b, j, s)
                assert hi[j * H + s] == [s + H + o[j]], (b, j, s)
            assert tail[4 * H + j] == [2 * H + o[j]], (b, j)
        assert len(lo) == 4 * H and len(tail) == 4


@pytest.mark.parametrize("S,MMAX", G.QUADS16)
@pytest.mark.parametrize("kind", [0, 1])
def test_quads_16bit(S, MMAX, kind):
    op = "f16" if kind == 0 else "bf16"
    nb_m = 8 * (MMAX + 1)
    for b, body in _blocks(G.emit_quad16(S, MMAX, kind)).items():
        r0, mb = b // nb_m, b % nb_m
        p = [r0 + o for o in G.quad_steps(mb)]
        word, half, acc = {}, {}, defaultdict(list)
        for ins in body:
            ld = _load_offsets(ins)
            if ld:
                word[ld[0]] = ld[1] // 4
                continue
            m = re.fullmatch(r"mov\.b32 \{(\w+), (\w+)\}, (\w+);", ins)
            if m:
                w = word[m.group(3)]
                half[m.group(1)], half[m.group(2)] = 2 * w, 2 * w + 1  # low half first
                continue
            m = re.fullmatch(rf"add\.rn\.f32\.{op} %(\d+), (\w+), %\1;", ins)
            assert m, ins
            acc[int(m.group(1))].append(half[m.group(2)])
        for j in range(4):
            for s in range(S):
                assert acc[j * S + s] == [p[j] + s], (b, j, s)


@pytest.mark.parametrize("S,MMAX", G.QUADS8)
def test_quads_8bit(S, MMAX):
    H = S // 2
    ne = 4 * H
    nb_m = 8 * (MMAX + 1)
    for b, body in _blocks(G.emit_quad8(S, MMAX)).items():
        r0, mb = b // nb_m, b % nb_m
        p = [r0 + o for o in G.quad_steps(mb)]
        word, acc = {}, defaultdict(list)
        for ins in body:
            ld = _load_offsets(ins)
            if ld:
                word[ld[0]] = ld[1] // 4
                continue
            m = re.fullmatch(r"add\.u32 %(\d+), %\1, (\w+);", ins)
            assert m, ins
            acc[int(m.group(1))].append(word[m.group(2)])
        for j in range(4):
            if p[j] % 2 == 0:
                # e[j][i]: the word holding trial j's outputs 2i, 2i + 1
                for i in range(H):
                    assert acc[j * H + i] == [p[j] // 2 + i], (b, j, i)
                assert all(not acc[ne + j * (H + 1) + i] for i in range(H + 1))
            else:
                # f[j][i]: the word holding its outputs 2i - 1, 2i
                for i in range(H + 1):
                    assert acc[ne + j * (H + 1) + i] == [(p[j] - 1) // 2 + i], (b, j, i)
                assert all(not acc[j * H + i] for i in range(H))


@pytest.mark.parametrize("S,OMAX", G.PAIRS)
def test_pairs_fp32(S, OMAX):
    for d, body in _blocks(G.emit_pair(S, OMAX)).items():
        reg, acc = {}, defaultdict(list)
        for ins in body:
            ld = _load_offsets(ins)
            if ld:
                reg[ld[0]] = ld[1] // 4
                continue
            m = re.fullmatch(r"add\.f32 %(\d+), %\1, (\w+);", ins)
            assert m, ins
            acc[int(m.group(1))].append(reg[m.group(2)])
        for s in range(S):
            assert acc[s] == [s] and acc[S + s] == [s + d], (d, s)


@pytest.mark.parametrize("S,OMAX", G.SHAPES)
def test_shifted_register_windows(S, OMAX):
    w0 = S + 1  # operand number of window register 0
    for o, body in _blocks(G.emit(S, OMAX)).items():
        acc = defaultdict(list)
        for ins in body:
            m = re.fullmatch(r"add\.f32 %(\d+), %\1, %(\d+);", ins)
            assert m, ins
            acc[int(m.group(1))].append(int(m.group(2)) - w0)
        for s in range(S):
            assert acc[s] == [o + s], (o, s)


def test_quad_steps_cover_every_pattern():
    """Block index m * 8 + bits: the trials' offsets grow by m or m + 1 per
    step; for each m the eight blocks give the eight patterns {m, m + 1}^3
    (the producer takes m = the smallest step of the quad)."""
    from itertools import product
    for m in range(10):
        pats = set()
        for bits in range(8):
            o = G.quad_steps(m * 8 + bits)
            assert o[0] == 0
            pats.add(tuple(o[j + 1] - o[j] for j in range(3)))
        assert pats == set(product((m, m + 1), repeat=3))


def _loop_blocks(text):
    """(prologue, {block index: [instruction, ...]}) of a function whose
    stage loop runs inside the assembly."""
    pro, out, cur = [], {}, None
    for raw in text.splitlines():
        m = re.match(r'\s*"(.*)\\n"\s*$', raw)
        if not m:
            continue
        ins = m.group(1).strip()
        lab = re.fullmatch(r"C(\d+):", ins)
        if lab:
            cur = int(lab.group(1))
            out[cur] = []
        elif ins == "CEND:":
            cur = None
        elif cur is not None:
            out[cur].append(ins)
        elif not ins.startswith((".reg", "tbl:", "{", "}")):
            pro.append(ins)
    return pro, out


@pytest.mark.parametrize("S,MMAX,NCONS,V", G.QUADS8T)
def test_quads_8bit_stage_loop(S, MMAX, NCONS, V):
    """Every block of the 8-bit quads with the stage loop inside the assembly
    adds the right words into the right accumulators (as emit_quad8's
    blocks), in the load order and add forms of its variant, and the loop
    visits the stage's channels in order, each once, for 1 to 4 channels."""
    first, alt = V == 3, V in (3, 4)
    H = S // 2
    ne = 4 * H + 4 * (H + 1)
    nb_m = 8 * (MMAX + 1)
    pro, blocks = _loop_blocks(G.emit_quad8t(S, MMAX, NCONS, V))
    assert pro == [f"mov.u32 ip, %{ne + 1};", "ld.shared.v2.u32 {ix, iy}, [ip];", "mov.u32 ci, 1;",
                   f"add.u32 ad, %{ne}, ix;", "LOOP:", f"setp.lt.u32 p, ci, %{ne + 2};", "brx.idx.uni iy, tbl;"]
    assert len(blocks) == 2 * nb_m
    for b, body in blocks.items():
        r0, mb = b // nb_m, b % nb_m
        p = [r0 + o for o in G.quad_steps(mb)]
        # the next channel's info first, the jump back to the loop last
        assert body[:2] == [f"@p add.u32 ip, ip, {16 * NCONS};", "ld.shared.v2.u32 {ix, iy}, [ip];"]
        assert body[-4:] == ["@!p bra.uni CEND;", "add.u32 ci, ci, 1;", f"add.u32 ad, %{ne}, ix;",
                             "bra.uni LOOP;"]
        word, acc, forms, seen_add = {}, defaultdict(list), defaultdict(int), False
        for ins in body[2:-4]:
            m = re.fullmatch(r"ld\.shared\.b32 (\w+), \[ad\+(\d+)\];", ins)
            if m:
                assert not (first and seen_add), "a load after the adds"
                word[m.group(1)] = int(m.group(2)) // 4
                continue
            m = re.fullmatch(r"(add\.u32|add\.u16x2) %(\d+), %\2, (\w+);", ins)
            assert m, ins
            seen_add = True
            forms[m.group(1)] += 1
            acc[int(m.group(2))].append(word[m.group(3)])
        if alt:
            assert abs(forms["add.u32"] - forms["add.u16x2"]) <= 1
        else:
            assert forms["add.u16x2"] == 0
        for j in range(4):
            if p[j] % 2 == 0:
                for i in range(H):
                    assert acc[j * H + i] == [p[j] // 2 + i], (b, j, i)
                assert all(not acc[4 * H + j * (H + 1) + i] for i in range(H + 1))
            else:
                for i in range(H + 1):
                    assert acc[4 * H + j * (H + 1) + i] == [(p[j] - 1) // 2 + i], (b, j, i)
                assert all(not acc[j * H + i] for i in range(H))
    # control flow, step by step as the prologue, LOOP and the block ends say
    g = __import__("numpy").random.default_rng(S + V)
    for nc in range(1, 5):
        base, sb = 4096, 100000
        info = {base + k * 16 * NCONS: (int(g.integers(0, 1 << 16)), int(g.integers(0, 2 * nb_m)))
                for k in range(4)}
        ip = base
        ix, iy = info[ip]
        ci, ad, visits = 1, sb + ix, []
        for _ in range(8):
            pred = ci < nc            # LOOP: setp
            visits.append((iy, ad))  # brx to block iy, which reads from ad
            if pred:
                ip += 16 * NCONS
            ix, iy = info[ip]
            if not pred:
                break
            ci += 1
            ad = sb + ix
        want = [(info[base + k * 16 * NCONS][1], sb + info[base + k * 16 * NCONS][0]) for k in range(nc)]
        assert visits == want, (nc, visits, want)
