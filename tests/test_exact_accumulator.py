"""The exact fixed-point accumulator of the CUDA reductions (acc_add / acc_round in
csrc/eptv_internal.cuh), compiled for the host with stand-ins for the CUDA intrinsics
(single-threaded: the device atomics become plain additions, which is what makes the
result order-independent), against exact rational sums: every total of FP32-derived
block partials must be the correctly rounded exact sum, including round-to-even ties,
cancellation, and the non-finite and overflow flags.  Values are spread over the
kAccCopies copies as blocks spread them (value i into copy i mod kAccCopies), and the
copies' words are added before rounding, as the device read-out does."""
import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1009_2288_b300", "csrc", "eptv_internal.cuh")

SHIMS = r'''
#include <cstdio>
#include <cstring>
#include <cmath>
#include <cstdlib>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double x) { long long r; memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; memcpy(&r, &x, 8); return r; }
static inline int __clz(unsigned int x) { return x ? __builtin_clz(x) : 32; }
static inline double __ull2double_rn(unsigned long long x) { return (double)x; }
static inline unsigned long long __ldcg(const unsigned long long *p) { return *p; }
static inline void atomicAdd(unsigned long long *p, unsigned long long v) { *p += v; }
static inline void atomicOr(unsigned long long *p, unsigned long long v) { *p |= v; }
static inline unsigned int __float_as_uint(float x) { unsigned int r; memcpy(&r, &x, 4); return r; }
static inline float __uint_as_float(unsigned int x) { float r; memcpy(&r, &x, 4); return r; }
'''

MAIN = r'''
int main() {
    unsigned long long acc[kAccCopies][kAccStride];
    memset(acc, 0, sizeof acc);
    char line[128];
    long n = 0;
    while (fgets(line, sizeof line, stdin)) {
        if (line[0] == 'E') {
            long long w[kAccChunks];
            unsigned long long flags = 0;
            for (int i = 0; i < kAccChunks; ++i) {
                w[i] = 0;
                for (int c = 0; c < kAccCopies; ++c) w[i] += (long long)acc[c][i];
            }
            for (int c = 0; c < kAccCopies; ++c) flags |= acc[c][kAccChunks];
            const double r = acc_round(w, flags);
            printf("%016llx\n", (unsigned long long)__double_as_longlong(r));
            memset(acc, 0, sizeof acc);
            n = 0;
            continue;
        }
        if (line[0] == 'F')        // an FP32 value added by acc_add_f32
            acc_add_f32(acc[n % kAccCopies], __uint_as_float((unsigned int)strtoul(line + 1, 0, 16)));
        else
            acc_add(acc[n % kAccCopies], __longlong_as_double((long long)strtoull(line, 0, 16)));
        ++n;
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def accumulator(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    src = open(HEADER).read()
    body = src[src.index("constexpr int kAccChunks"):src.index("// All NT threads of a block (NT a multiple of 32)")]
    d = tmp_path_factory.mktemp("acc")
    cpp, exe = d / "acc.cpp", d / "acc"
    cpp.write_text(SHIMS + body + MAIN)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", str(exe), str(cpp)])

    def run(groups, as_f32=False):
        lines = []
        for g in groups:
            if as_f32:
                lines += ["F%08x" % struct.unpack("<I", struct.pack("<f", x))[0] for x in g] + ["E"]
            else:
                lines += ["%016x" % struct.unpack("<Q", struct.pack("<d", x))[0] for x in g] + ["E"]
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split()
        return [struct.unpack("<d", struct.pack("<Q", int(h, 16)))[0] for h in out]
    return run


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def test_sums_of_fp32_partials_are_correctly_rounded(accumulator):
    rng = random.Random(7)
    groups = []
    for _ in range(300):
        n = rng.choice([1, 2, 5, 64, 1024])
        scale = 2.0 ** rng.randint(-140, 120)
        vals = [f32(rng.uniform(-1, 1) * scale * 2.0 ** rng.randint(-20, 5)) for _ in range(n)]
        if rng.random() < 0.3:
            vals = [abs(v) for v in vals]
        parts = []
        for i in range(0, n, 4):          # block partials: FP64 sums of FP32 warp sums
            s = 0.0
            for v in vals[i:i + 4]:
                s += v
            parts.append(s)
        groups.append(parts)
    got = accumulator(groups)
    for g, r in zip(groups, got):
        assert r == float(sum(Fraction(x) for x in g)), g[:3]


def test_order_does_not_matter(accumulator):
    rng = random.Random(3)
    g = [f32(rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)) for _ in range(500)]
    perms = [g, list(reversed(g)), sorted(g), rng.sample(g, len(g))]
    got = accumulator(perms)
    assert len(set(got)) == 1
    assert got[0] == float(sum(Fraction(x) for x in g))


def test_ties_cancellation_and_special_values(accumulator):
    cases = [
        ([2.0 ** 53, 1.0], 2.0 ** 53),                   # tie -> even
        ([2.0 ** 53, 1.0, 2.0 ** -100], 2.0 ** 53 + 2),  # just above the tie
        ([2.0 ** 53 + 2, 1.0], 2.0 ** 53 + 4),           # tie -> even (upwards)
        ([-(2.0 ** 53), -1.0], -(2.0 ** 53)),
        ([1e30, -1e30, 3.0], 3.0),                       # exact cancellation
        ([1.0, 2.0 ** -149 * 3, -1.0], 2.0 ** -149 * 3),
        ([2.0 ** -149], 2.0 ** -149),
        ([0.0, -0.0], 0.0),
        ([], 0.0),
        ([3.4e38, 3.4e38, 3.4e38], 3.0 * 3.4e38),
    ]
    got = accumulator([c for c, _ in cases])
    for (c, want), r in zip(cases, got):
        assert r == want, c
    inf, nan = float("inf"), float("nan")
    sp = accumulator([[inf, 1.0], [-inf, 2.0], [inf, -inf], [nan, 1.0], [2.0 ** 200], [-(2.0 ** 195)]])
    assert sp[0] == inf and sp[1] == -inf
    assert math.isnan(sp[2]) and math.isnan(sp[3])
    assert sp[4] == inf and sp[5] == -inf              # beyond the accumulator's range


def test_fp32_values_added_directly(accumulator):
    """acc_add_f32 (integer atomics only): sums of FP32 warp sums, including subnormals,
    both signs, cancellation and FLT_MAX, are the correctly rounded exact sums and equal the
    FP64 path's; non-finite values set the flags."""
    rng = random.Random(11)
    groups = []
    for _ in range(300):
        n = rng.choice([1, 3, 32, 500])
        scale = 2.0 ** rng.randint(-149, 100)
        groups.append([f32(rng.uniform(-1, 1) * scale * 2.0 ** rng.randint(-24, 24)) for _ in range(n)])
    groups += [[2.0 ** -149, -(2.0 ** -149)], [f32(1.1754942e-38), 2.0 ** -149], [f32(3.4028235e38)] * 3,
               [f32(16777217.0), 1.0, -16777216.0], [-0.0], []]
    got = accumulator(groups, as_f32=True)
    want64 = accumulator(groups)
    for g, r, r64 in zip(groups, got, want64):
        assert r == float(sum(Fraction(x) for x in g)), g[:3]
        assert r == r64
    inf, nan = float("inf"), float("nan")
    sp = accumulator([[inf, 1.0], [-inf, 2.0], [nan]], as_f32=True)
    assert sp[0] == inf and sp[1] == -inf and math.isnan(sp[2])
