"""Host checks of the double-float header used by the FP64-accurate stencil
kernels (paper_2103_01874_gb300/csrc/dfloat.cuh): the integer-based FP64 <->
pair conversions and the pair arithmetic, against exact rational arithmetic.
The header is plain integer/IEEE-float code, compiled here with g++
(-ffp-contract=off) exactly as nvcc compiles it for the device."""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction as Q

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_01874_gb300", "csrc")
EPS48 = Q(1, 2 ** 48)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("dfh") / "dfh")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(ROOT, "tests", "dfloat_harness.cpp"), "-o", exe], check=True)

    def run(lines):
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        return out.stdout.split("\n")[: len(lines)]
    return run


def f32(x):
    return struct.unpack("f", struct.pack("f", x))[0]


def samples(n=4000, seed=0):
    rng = random.Random(seed)
    xs = [0.0, -0.0, 1.0, -1.0, 2.0, 0.5, 3.0, 1e-20, -7.25e13, 6.02e23, 2.0 ** -70, 2.0 ** 100,
          1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, 1.0 - 2.0 ** -53, -(1.0 - 2.0 ** -53)]
    for _ in range(n):
        m = rng.uniform(1.0, 2.0)
        e = rng.randint(-60, 90)
        xs.append(rng.choice((-1, 1)) * m * 2.0 ** e)
    return xs


def test_d2df_exactness(harness):
    xs = samples()
    out = harness([f"d2df {x.hex()}" for x in xs])
    for x, line in zip(xs, out):
        hi, lo = (float.fromhex(t) for t in line.split())
        assert hi == f32(hi) and lo == f32(lo)
        err = abs(Q(hi) + Q(lo) - Q(x))
        assert err <= EPS48 * abs(Q(x)), (x, hi, lo)


@pytest.mark.parametrize("conv", ["df2d", "df2d_alu"])
def test_df2d_roundtrip(harness, conv):
    xs = samples(seed=1)
    pairs = harness([f"d2df {x.hex()}" for x in xs])
    back = harness([f"{conv} {p}" for p in pairs])
    for x, p, b in zip(xs, pairs, back):
        hi, lo = (float.fromhex(t) for t in p.split())
        y = float.fromhex(b)
        exact = Q(hi) + Q(lo)
        # faithful: within one double ulp of the pair's exact value
        assert abs(Q(y) - exact) <= Q(2) ** -52 * abs(exact), (x, hi, lo, y)
        assert abs(Q(y) - Q(x)) <= EPS48 * abs(Q(x))


@pytest.mark.parametrize("conv", ["df2d", "df2d_alu"])
def test_df2d_power_of_two_borrow(harness, conv):
    """A negative lo below a power-of-two hi counts in the lower binade."""
    cases = []
    for e in (-20, 0, 7, 40):
        h = 2.0 ** e
        for lo in (-h * 2.0 ** -26, -h * 2.0 ** -30, h * 2.0 ** -26, -h * 3 * 2.0 ** -27):
            cases.append((h, f32(lo)))
            cases.append((-h, -f32(lo)))
    out = harness([f"{conv} {h.hex()} {lo.hex()}" for h, lo in cases])
    for (h, lo), line in zip(cases, out):
        y = float.fromhex(line)
        exact = Q(h) + Q(lo)
        assert abs(Q(y) - exact) <= Q(2) ** -52 * abs(exact), (h, lo, y)


@pytest.mark.parametrize("op", ["add", "sub", "mul", "mulf", "recip"])
def test_pair_arithmetic(harness, op):
    rng = random.Random(hash(op) & 0xFFFF)
    lines, args = [], []
    for _ in range(1500):
        a = rng.uniform(-1e4, 1e4) if op != "recip" else rng.uniform(1.0, 2000.0)
        b = rng.uniform(-1e4, 1e4)
        if op in ("add", "sub") and rng.random() < 0.3:
            b = (-a if op == "add" else a) * (1 + rng.uniform(-1e-6, 1e-6))  # cancellation
        pa = harness_pair(a)
        pb = harness_pair(b) if op != "mulf" else (f32(b), 0.0)
        args.append((pa, pb))
        lines.append(f"{op} {pa[0].hex()} {pa[1].hex()} {pb[0].hex()} {pb[1].hex()}")
    out = harness(lines)
    for (pa, pb), line in zip(args, out):
        hi, lo = (float.fromhex(t) for t in line.split())
        A = Q(pa[0]) + Q(pa[1])
        B = Q(pb[0]) + Q(pb[1])
        want = {"add": A + B, "sub": A - B, "mul": A * B, "mulf": A * B, "recip": 1 / A}[op]
        got = Q(hi) + Q(lo)
        if op in ("add", "sub"):
            bound = Q(2) ** -46 * (abs(A) + abs(B))   # absolute, scaled by the operands
        else:
            bound = Q(2) ** -45 * abs(want)
        assert abs(got - want) <= bound, (op, pa, pb, hi, lo)


@pytest.mark.parametrize("op", ["dot2sub", "dot2add"])
def test_fused_pair_dot_product(harness, op):
    """dd_dot2 (the pair complex multiply's components): a b -+ c d of four
    pairs, exact rationals; bounded by 2^-45 of |a b| + |c d| (products of
    near-equal size cancel: the bound is on the operands, like the adds')."""
    rng = random.Random(7 if op == "dot2sub" else 8)
    lines, args = [], []
    for _ in range(1500):
        xs = [rng.uniform(-1e3, 1e3) for _ in range(4)]
        if rng.random() < 0.3:  # a b close to c d (or to -c d)
            xs[2] = xs[0] * (1 + rng.uniform(-1e-6, 1e-6))
            xs[3] = (xs[1] if op == "dot2sub" else -xs[1]) * (1 + rng.uniform(-1e-6, 1e-6))
        ps = [harness_pair(x) for x in xs]
        args.append(ps)
        lines.append(op + " " + " ".join(f"{p[0].hex()} {p[1].hex()}" for p in ps))
    out = harness(lines)
    for ps, line in zip(args, out):
        hi, lo = (float.fromhex(t) for t in line.split())
        A, B, C, D = (Q(p[0]) + Q(p[1]) for p in ps)
        want = A * B - C * D if op == "dot2sub" else A * B + C * D
        got = Q(hi) + Q(lo)
        assert abs(got - want) <= Q(2) ** -45 * (abs(A * B) + abs(C * D)), (op, ps, hi, lo)
        assert abs(Q(lo)) <= Q(2) ** -23 * abs(Q(hi)) or hi == 0.0, "normalised"


def test_lazy_adds_then_normalise(harness):
    """Two lazy adds (no renormalisation between) and one dd_norm: the sum to
    2^-45 of the operands' magnitudes, and a normalised result."""
    rng = random.Random(11)
    lines, args = [], []
    for _ in range(1500):
        xs = [rng.uniform(-1e4, 1e4) for _ in range(3)]
        if rng.random() < 0.3:
            xs[1] = -xs[0] * (1 + rng.uniform(-1e-6, 1e-6))
        ps = [harness_pair(x) for x in xs]
        args.append(ps)
        lines.append("addlazy " + " ".join(f"{p[0].hex()} {p[1].hex()}" for p in ps))
    out = harness(lines)
    for ps, line in zip(args, out):
        hi, lo = (float.fromhex(t) for t in line.split())
        A, B, C = (Q(p[0]) + Q(p[1]) for p in ps)
        got = Q(hi) + Q(lo)
        assert abs(got - (A + B + C)) <= Q(2) ** -45 * (abs(A) + abs(B) + abs(C)), (ps, hi, lo)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 7, 8, 9, 12, 16, 24, 25, 48, 96, 128, 129, 193, 255, 256, 257,
                               384, 385, 513, 1025, 65536, 65537, 1 << 20, (1 << 20) + 3])
def test_fastdiv_exact(harness, d):
    """Magic-number division equals integer division for 0 <= x < 2^31."""
    lines = [f"fastdiv {d} 0 200000 1", f"fastdiv {d} 0 200000 10007", f"fastdiv {d} 2147000000 483647 1",
             f"fastdiv {d} {max(0, d * 1000 - 5)} 100 1"]
    assert harness(lines) == ["0"] * 4


def harness_pair(x):
    """A normalised pair for x (computed here, independent of the header)."""
    hi = f32(x)
    lo = f32(x - hi)
    return hi, lo
