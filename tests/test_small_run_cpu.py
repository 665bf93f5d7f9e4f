"""Launch arithmetic of the one-launch run of small binary graphs, checked on the host.

The launcher (launch_lr_small_run) sizes one block, or a cluster of C blocks, from the
variable count V and the factor count F; the kernels index shared memory, and through
distributed shared memory other blocks' shared memory, from that sizing. This restates
the sizing and the kernels' index formulas and checks, over a sweep of sizes up to the
limits, that every variable and every factor is owned by exactly one thread, that every
slot of the 4-slot layout maps to a block of the cluster and an offset inside its shared
memory, and that block sizes stay within 1,024 threads -- the facts a launch relies on to
stay in bounds.
"""
import numpy as np
import pytest

THREADS = 1024  # kLrSmallThreads
BLOCK_V, BLOCK_F = 1024, 2048  # kLrSmallMaxV, kLrSmallMaxF


def block_shape(V, F):
    one = F <= THREADS
    per = max(V, F) if one else max(V, (F + 1) // 2)
    return max(32, (per + 31) // 32 * 32), 1 if one else 2


def cluster_shape(V, F, C):
    Vc, Fc = -(-V // C), -(-F // C)
    one = Fc <= THREADS
    per = max(Vc, Fc) if one else max(Vc, (Fc + 1) // 2)
    return max(32, (per + 31) // 32 * 32), 1 if one else 2, Vc, Fc


def slot_home(p, V, Vc):
    k = int(p >= V) + int(p >= 2 * V) + int(p >= 3 * V)
    v = p - k * V
    rank = v // Vc
    lv = v - rank * Vc
    return rank, k * Vc + lv, lv


@pytest.mark.parametrize("V,F", [(1, 0), (2, 1), (4, 4), (100, 180), (700, 1300), (1024, 1023), (1024, 1984),
                                 (1000, 2048)])
def test_block_owns_every_item_once(V, F):
    nt, NF = block_shape(V, F)
    assert nt <= THREADS and nt % 32 == 0
    assert V <= nt  # thread t owns variable t
    owned = [t + j * nt for t in range(nt) for j in range(NF) if t + j * nt < F]
    assert sorted(owned) == list(range(F))
    # shared memory: V float2 of totals then 4 V floats of slots (24 V bytes)
    assert 24 * V <= 48 * 1024


@pytest.mark.parametrize("C", [8, 16])
def test_cluster_partition_and_slot_homes(C):
    rng = np.random.default_rng(C)
    sizes = [(2, 1), (9, 8), (C * 1024, C * 1024 - 1), (C * 1024, C * 2048), (701, 1351), (4096, 8064)]
    sizes += [(int(v), int(rng.integers(v // 2, min(2 * v, C * BLOCK_F) + 1)))
              for v in rng.integers(700, C * BLOCK_V + 1, 40)]
    for V, F in sizes:
        if V > C * BLOCK_V or F > C * BLOCK_F:
            continue
        nt, NF, Vc, Fc = cluster_shape(V, F, C)
        assert nt <= THREADS and nt % 32 == 0
        assert Vc <= nt and Vc <= BLOCK_V and 24 * Vc <= 48 * 1024
        # variables: block r owns r Vc .. min(V, (r + 1) Vc) - 1, thread t the t-th of them
        vars_owned = [r * Vc + t for r in range(C) for t in range(max(0, min(Vc, V - r * Vc)))]
        assert sorted(vars_owned) == list(range(V))
        # factors: block r owns r Fc + i for i < Fc, thread t the items t + j nt
        fac_owned = [r * Fc + t + j * nt for r in range(C) for t in range(nt) for j in range(NF)
                     if t + j * nt < Fc and r * Fc + t + j * nt < F]
        assert sorted(fac_owned) == list(range(F))
        # every slot of the 4-slot layout has a home block and an offset inside its 4 Vc
        # floats of d (and its variable inside its Vc totals)
        for p in list(range(0, 4 * V, max(1, V // 7))) + [4 * V - 1, V - 1, V, 3 * V]:
            rank, off, lv = slot_home(p, V, Vc)
            assert 0 <= rank < C and 0 <= off < 4 * Vc and 0 <= lv < Vc
        # a thread with no factor reads slot 0's home: block 0, which owns variable 0
        assert slot_home(0, V, Vc)[0] == 0
        # unpack: block r writes the edges of its factors, 2 r Fc .. 2 min(F, (r + 1) Fc) - 1
        edges = [e for r in range(C) for e in range(2 * r * Fc, 2 * min(F, (r + 1) * Fc))]
        assert sorted(edges) == list(range(2 * F))
