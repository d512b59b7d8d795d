"""The kernel planner's rule (csrc/umi_plan.cu) against a restatement of it,
over a grid of window lengths and band sizes.  Host logic only: without a GPU
the library sizes plans for a device of one SM, with one the device's own SM
count is used, and the restatement takes the same count.

The rule: a band is in the latency regime when its throughput variant yields
fewer than 32 tiles per SM at the shortest chain; throughput bands take the
smallest covering slot capacity (below 5e5 positions the tight fit with the
largest register budget), latency bands a 32-lane variant within 2W; the
chain gives about 16 warps per SM a tile (8 for one- and two-lane latency
bands), capped at 136 (groups of 8 or more lanes) or 33 positions; CTAs have
128 threads below 3e5 positions, else 256 for groups wider than two lanes."""
import os
import re

import pytest

from paper_2604_06602_gb300 import build as libbuild
from paper_2604_06602_gb300 import umi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def variant_table():
    text = open(os.path.join(ROOT, "paper_2604_06602_gb300", "csrc", "umi_variants.h")).read()
    body = text[text.index("#define UMI_VARIANT_LIST(X)"):]
    body = body[:body.index("\n\n")] if "\n\n" in body else body
    out = [tuple(int(v) for v in m.groups()) for m in re.finditer(r"X\((\d+),\s*(\d+),\s*(\d+)\)", body)]
    assert len(out) >= 10
    return out


def sm_count():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_properties(0).multi_processor_count
    except ImportError:
        pass
    return 1


def chain_at_least(G, target):
    target = min(max(target, 1), 1 << 20)
    if G >= 32:
        return target
    odd = -(-target // G)
    if odd % 2 == 0:
        odd += 1
    return G * odd


def chain_cap(G):
    return chain_at_least(G, 136 if G >= 8 else 33)


class Rule:
    def __init__(self, table, sms):
        self.t = table
        self.sms = max(1, sms)

    def smallest(self, W):
        return min(G * R for G, R, _ in self.t if G * R >= W)

    def tight(self, v, W):
        S = v[0] * v[1]
        return S >= W and (S == self.smallest(W) or 3 * S <= 4 * W)

    def throughput_variant(self, W, P):
        rich = 0 < P < 500000
        best = None
        for i, v in enumerate(self.t):
            if not self.tight(v, W):
                continue
            if best is None:
                best = i
                continue
            a, b = v, self.t[best]
            Sa, Sb = a[0] * a[1], b[0] * b[1]
            if (a[2] < b[2] or (a[2] == b[2] and Sa < Sb)) if rich else Sa < Sb:
                best = i
        return best

    def latency_variant(self, W, P):
        smallest = self.smallest(W)
        best = None
        for i, v in enumerate(self.t):
            S = v[0] * v[1]
            if v[0] != 32 or S < W or (S != smallest and S > 2 * W):
                continue
            if best is None:
                best = i
                continue
            b = self.t[best]
            ta, tb = self.tight(v, W), self.tight(b, W)
            if ta != tb:
                if ta:
                    best = i
                continue
            if v[2] != b[2]:
                if v[2] < b[2]:
                    best = i
                continue
            if S < b[0] * b[1]:
                best = i
        return best if best is not None else self.throughput_variant(W, P)

    def regime(self, W, P):
        if P <= 0:
            return 0
        G = self.t[self.throughput_variant(W, P)][0]
        tile = (32 // G) * (1 if G >= 32 else G)
        items = -(-P // tile)
        return 1 if items < 32 * self.sms else 0

    def chain_for(self, G, P, regime):
        target = 8 if (regime == 1 and G <= 2) else 16
        warps = self.sms * target
        per_warp = -(-P // warps)
        return chain_at_least(G, -(-(per_warp * G) // 32))

    def plan(self, W, P):
        regime = self.regime(W, P)
        v = self.latency_variant(W, P) if regime == 1 else self.throughput_variant(W, P)
        G, R, _ = self.t[v]
        threads = 128 if (0 < P < 300000 or G <= 2) else 256
        chain = chain_cap(G)
        if P > 0:
            chain = min(chain, min(chain_cap(G), self.chain_for(G, P, regime)))
        return {"lanes": G, "slots": R, "chain": chain, "threads": threads, "variant": v, "latency": regime}


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    lib = umi.load()
    umi.clear_tuning()
    return lib


WINDOWS = [1, 3, 7, 9, 15, 17, 25, 27, 31, 33, 63, 65, 121, 127, 129, 191, 193, 217, 361, 367, 369, 383,
           385, 721, 767, 769, 1025, 1535, 1537, 2161, 2175, 2177, 4095]
SIZES = [1, 31, 32, 33, 500, 4_000, 12_500, 37_000, 155_647, 155_648, 299_999, 300_000, 499_999,
         500_000, 3_000_000, 18_000_000, 30_208_000]


@pytest.mark.parametrize("W", WINDOWS)
def test_plan_follows_rule(lib, W):
    rule = Rule(variant_table(), sm_count())
    for P in SIZES:
        assert umi.get_plan(W, P) == rule.plan(W, P), (W, P)


def test_plan_invariants(lib):
    """Every plan covers W, uses a bank-conflict-free chain, and stays within
    the chain cap, over every odd W up to the largest window."""
    table = variant_table()
    for W in range(1, umi.max_window() + 1, 2):
        for P in (1000, 1_000_000):
            p = umi.get_plan(W, P)
            G, R = p["lanes"], p["slots"]
            assert (G, R) == table[p["variant"]][:2]
            assert G * R >= W
            assert p["chain"] >= 1 and p["chain"] <= chain_cap(G)
            if G < 32:
                assert p["chain"] % G == 0 and (p["chain"] // G) % 2 == 1
            assert p["threads"] in (128, 256)


def test_bad_windows_rejected(lib):
    for W in (0, 2, 4096, umi.max_window() + 2, -1):
        with pytest.raises(umi.UmiError) as e:
            umi.get_plan(W, 1000)
        assert e.value.status == umi.UMI_ERR_INVALID_ARG
