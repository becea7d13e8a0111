"""The double-float primitives of the DF outer iteration (csrc/df.cuh), built
for the host with g++ (no FP contraction) and checked against exact rational
arithmetic:

* TwoSum and the FMA product are error-free: s + e == a + b and p + e == a b
  exactly, for random FP32 operands of mixed signs and exponents.
* FastTwoSum is error-free when |a| >= |b|.
* df_add / df_sub / df_add_f / df_mul / df_mul_f return normalised pairs
  (|lo| <= ulp(hi) / 2) within a few units of 2^-48 of the exact result,
  including sums that cancel to a few bits.
* df_from_double / df_to_double round-trip an FP64 value to within 2^-48.
* The cheaper forms used where sums do not cancel -- df_add_fast, the
  product accumulators df_acc_prod / df_acc_prod_f, and the stencil value
  D z - (v1 + ... + v6) by cascaded summation (Sum2) -- are within a few units
  of 2^-48 of the sum of the magnitudes of their terms.
"""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2204_06083_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <cmath>
#include "df.cuh"
using namespace ebk;
static float f(uint32_t u) { float v; std::memcpy(&v, &u, 4); return v; }
static uint32_t u(float v) { uint32_t r; std::memcpy(&r, &v, 4); return r; }
static uint64_t ud(double v) { uint64_t r; std::memcpy(&r, &v, 8); return r; }
int main() {
  char op[16];
  unsigned a, b, c, d;
  unsigned long long dv;
  while (std::scanf("%15s", op) == 1) {
    if (!std::strcmp(op, "d")) {  // double round trip
      std::scanf("%llx", &dv);
      double x;
      std::memcpy(&x, &dv, 8);
      DF r = df_from_double(x);
      std::printf("%08x %08x %016llx\n", u(r.hi), u(r.lo), (unsigned long long)ud(df_to_double(r)));
      continue;
    }
    if (!std::strcmp(op, "accp") || !std::strcmp(op, "accpf")) {  // s += a b
      unsigned v[6];
      for (int i = 0; i < 6; ++i) std::scanf("%x", &v[i]);
      DF s{f(v[0]), f(v[1])};
      if (op[4] == 'f') df_acc_prod_f(s, DF{f(v[2]), f(v[3])}, f(v[4]));
      else df_acc_prod(s, DF{f(v[2]), f(v[3])}, DF{f(v[4]), f(v[5])});
      std::printf("%08x %08x\n", u(s.hi), u(s.lo));
      continue;
    }
    if (!std::strcmp(op, "st")) {  // D z - (v1 + ... + v6), D = (dh, dl)
      unsigned v[9];
      for (int i = 0; i < 9; ++i) std::scanf("%x", &v[i]);
      Sum2 sm = sum2_start(f(v[3]));
      for (int i = 4; i < 9; ++i) sum2_add(sm, f(v[i]));
      float p, pe;
      two_prod(f(v[0]), f(v[2]), p, pe);
      pe = std::fma(f(v[1]), f(v[2]), pe);
      DF r = df_prod_minus_sum2(p, pe, sm);
      std::printf("%08x %08x\n", u(r.hi), u(r.lo));
      continue;
    }
    std::scanf("%x %x %x %x", &a, &b, &c, &d);
    float s, e;
    DF r{0.f, 0.f};
    const DF x{f(a), f(b)}, y{f(c), f(d)};
    if (!std::strcmp(op, "ts")) { two_sum(f(a), f(c), s, e); r = DF{s, e}; }
    else if (!std::strcmp(op, "fts")) { fast_two_sum(f(a), f(c), s, e); r = DF{s, e}; }
    else if (!std::strcmp(op, "tp")) { two_prod(f(a), f(c), s, e); r = DF{s, e}; }
    else if (!std::strcmp(op, "add")) r = df_add(x, y);
    else if (!std::strcmp(op, "addfast")) r = df_add_fast(x, y);
    else if (!std::strcmp(op, "sub")) r = df_sub(x, y);
    else if (!std::strcmp(op, "addf")) r = df_add_f(x, f(c));
    else if (!std::strcmp(op, "mul")) r = df_mul(x, y);
    else if (!std::strcmp(op, "mulf")) r = df_mul_f(x, f(c));
    std::printf("%08x %08x\n", u(r.hi), u(r.lo));
  }
  return 0;
}
"""


def _bits(v):
    return struct.unpack("<I", struct.pack("<f", v))[0]


def _flt(b):
    return struct.unpack("<f", struct.pack("<I", b))[0]


def _fr(v):
    return Fraction(v)


def _ulp(v):
    if v == 0.0:
        return Fraction(0)
    m, e = __import__("math").frexp(abs(v))
    return Fraction(2) ** (e - 24)


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("df")
    src = d / "df_check.cpp"
    src.write_text(PROG)
    exe = d / "df_check"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    return str(exe)


def _run(prog, lines):
    out = subprocess.run([prog], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    return [tuple(int(t, 16) for t in l.split()) for l in out.strip().splitlines()]


def _rand_f32(rng, lo=-20, hi=20):
    m = rng.uniform(1.0, 2.0) * (1 if rng.random() < 0.5 else -1)
    return _flt(_bits(float(m) * 2.0 ** rng.randint(lo, hi)))


def _rand_df(rng):
    hi = _rand_f32(rng)
    lo = _flt(_bits(rng.uniform(-0.5, 0.5) * float(_ulp(hi))))
    return hi, lo


def _norm_ok(hi, lo):
    return abs(_fr(lo)) <= _ulp(hi) / 2


def test_error_free_transformations(prog):
    rng = random.Random(7)
    cases, want = [], []
    for _ in range(3000):
        a, b = _rand_f32(rng), _rand_f32(rng)
        if rng.random() < 0.2:  # near cancellation
            b = -_flt(_bits(a) ^ rng.randint(0, 7))
        for op in ("ts", "tp"):
            cases.append(f"{op} {_bits(a):x} 0 {_bits(b):x} 0")
            want.append((op, a, b))
        big, small = (a, b) if abs(a) >= abs(b) else (b, a)
        cases.append(f"fts {_bits(big):x} 0 {_bits(small):x} 0")
        want.append(("fts", big, small))
    for (op, a, b), (s, e) in zip(want, _run(prog, cases)):
        exact = _fr(a) + _fr(b) if op != "tp" else _fr(a) * _fr(b)
        assert _fr(_flt(s)) + _fr(_flt(e)) == exact, (op, a, b)


def _check_df(prog, op, xs, ys, exact_fn, ulps=8):
    lines = [f"{op} {_bits(x[0]):x} {_bits(x[1]):x} {_bits(y[0]):x} {_bits(y[1]):x}" for x, y in zip(xs, ys)]
    worst = 0.0
    for x, y, (h, l) in zip(xs, ys, _run(prog, lines)):
        hi, lo = _flt(h), _flt(l)
        exact = exact_fn(_fr(x[0]) + _fr(x[1]), _fr(y[0]) + _fr(y[1]))
        got = _fr(hi) + _fr(lo)
        assert _norm_ok(hi, lo), (op, x, y, hi, lo)
        if exact != 0:
            err = abs(got - exact) / abs(exact)
            worst = max(worst, float(err))
            assert err <= ulps * Fraction(2) ** -48, (op, x, y, float(err))
        else:
            assert got == 0
    return worst


def test_df_operations_accuracy(prog):
    rng = random.Random(11)
    n = 2000
    xs = [_rand_df(rng) for _ in range(n)]
    ys = [_rand_df(rng) for _ in range(n)]
    # sums whose high parts cancel (the residual update r - alpha q at convergence)
    for i in range(0, n, 5):
        ys[i] = (-xs[i][0], _flt(_bits(rng.uniform(-0.5, 0.5) * float(_ulp(xs[i][0])))))
    _check_df(prog, "add", xs, ys, lambda a, b: a + b)
    _check_df(prog, "sub", xs, ys, lambda a, b: a - b)
    _check_df(prog, "mul", xs, ys, lambda a, b: a * b)
    ysf = [(y[0], 0.0) for y in ys]
    _check_df(prog, "addf", xs, ysf, lambda a, b: a + b)
    _check_df(prog, "mulf", xs, ysf, lambda a, b: a * b)


def test_df_cancellation_to_few_bits(prog):
    """x + y where x and y agree in all but their last few bits: df_add keeps
    the low parts, so the result is exact (the FP32 sum of the high parts alone
    would lose everything below them)."""
    rng = random.Random(3)
    xs, ys = [], []
    for _ in range(500):
        hi = _rand_f32(rng)
        lo1 = _flt(_bits(rng.uniform(-0.5, 0.5) * float(_ulp(hi))))
        lo2 = _flt(_bits(rng.uniform(-0.5, 0.5) * float(_ulp(hi))))
        xs.append((hi, lo1))
        ys.append((-hi, lo2))
    lines = [f"add {_bits(x[0]):x} {_bits(x[1]):x} {_bits(y[0]):x} {_bits(y[1]):x}" for x, y in zip(xs, ys)]
    for x, y, (h, l) in zip(xs, ys, _run(prog, lines)):
        assert _fr(_flt(h)) + _fr(_flt(l)) == _fr(x[1]) + _fr(y[1])


def test_df_double_round_trip(prog):
    rng = random.Random(5)
    vals = [rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60) for _ in range(1000)] + [0.0, 1.0, -3.5]
    lines = ["d " + format(struct.unpack("<Q", struct.pack("<d", v))[0], "x") for v in vals]
    for v, (h, l, back) in zip(vals, _run(prog, lines)):
        hi, lo = _flt(h), _flt(l)
        assert _norm_ok(hi, lo)
        got = struct.unpack("<d", struct.pack("<Q", back))[0]
        if v != 0.0:
            assert abs(_fr(hi) + _fr(lo) - _fr(v)) <= abs(_fr(v)) * Fraction(2) ** -48
            assert abs(got - v) <= abs(v) * 2.0 ** -48
        else:
            assert got == 0.0


def _within(got, exact, mag, ulps=8):
    return abs(got - exact) <= ulps * Fraction(2) ** -48 * mag


def test_cheap_forms_accuracy(prog):
    rng = random.Random(19)
    n = 1500
    xs = [_rand_df(rng) for _ in range(n)]
    ys = [_rand_df(rng) for _ in range(n)]
    lines = [f"addfast {_bits(x[0]):x} {_bits(x[1]):x} {_bits(y[0]):x} {_bits(y[1]):x}" for x, y in zip(xs, ys)]
    for x, y, (h, l) in zip(xs, ys, _run(prog, lines)):
        a, b = _fr(x[0]) + _fr(x[1]), _fr(y[0]) + _fr(y[1])
        assert _norm_ok(_flt(h), _flt(l))
        assert _within(_fr(_flt(h)) + _fr(_flt(l)), a + b, abs(a) + abs(b))
    ss = [_rand_df(rng) for _ in range(n)]
    lines, want = [], []
    for s_, x, y in zip(ss, xs, ys):
        lines.append("accp " + " ".join(format(_bits(v), "x") for v in (s_[0], s_[1], x[0], x[1], y[0], y[1])))
        want.append((s_, x, y, False))
        lines.append("accpf " + " ".join(format(_bits(v), "x") for v in (s_[0], s_[1], x[0], x[1], y[0], 0.0)))
        want.append((s_, x, (y[0], 0.0), True))
    for (s_, x, y, _), (h, l) in zip(want, _run(prog, lines)):
        sv, a, b = _fr(s_[0]) + _fr(s_[1]), _fr(x[0]) + _fr(x[1]), _fr(y[0]) + _fr(y[1])
        assert _within(_fr(_flt(h)) + _fr(_flt(l)), sv + a * b, abs(sv) + abs(a * b))
    # the stencil value: D z - sum of six neighbours, with cancellation
    lines, want = [], []
    for _ in range(n):
        z = _rand_f32(rng, -3, 3)
        dh = 6.0 if rng.random() < 0.5 else _flt(_bits(rng.uniform(2.0, 6.0)))
        dl = 0.0 if dh == 6.0 else _flt(_bits(rng.uniform(-0.5, 0.5) * float(_ulp(dh))))
        nb = [_flt(_bits(z * rng.uniform(0.9, 1.1))) for _ in range(6)]
        lines.append("st " + " ".join(format(_bits(v), "x") for v in [dh, dl, z] + nb))
        want.append((dh, dl, z, nb))
    for (dh, dl, z, nb), (h, l) in zip(want, _run(prog, lines)):
        exact = (_fr(dh) + _fr(dl)) * _fr(z) - sum(_fr(v) for v in nb)
        mag = abs((_fr(dh) + _fr(dl)) * _fr(z)) + sum(abs(_fr(v)) for v in nb)
        assert _norm_ok(_flt(h), _flt(l))
        assert _within(_fr(_flt(h)) + _fr(_flt(l)), exact, mag), (dh, dl, z, nb)
