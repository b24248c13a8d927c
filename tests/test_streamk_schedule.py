"""Invariants of the stream-K schedule of the mode-product kernel, checked on
the CPU with the kernel's index arithmetic written out in Python.

With G CTAs and U work units of L = npair * kit iterations (unit, tile h of
the unit, K chunk), the first dp = (U / G - 1) G units (0 below two waves)
run whole, unit b + i G on CTA b; the Q = (U - dp) L iterations of the rest
are cut into G contiguous ranges [b Q / G, (b + 1) Q / G).  A unit touched
by several CTAs is finished by the last of them to deliver a partial; the
finisher sums the partial slots of each tile in CTA order.  The GPU parity
tests run the device code itself; this test pins the schedule it follows:
every iteration is computed exactly once, the delivery count the finisher
waits for is the number of partials written, the finisher finds exactly the
slots the writers used, no slot is written twice, and a CTA finishes at most
the two units at the ends of its range (the kernel keeps two)."""
import random

import pytest


def dp_units(units, G):
    w = units // G
    return (w - 1) * G if w >= 2 else 0


def owner(Q, q, G):
    # the CTA whose range [b Q / G, (b + 1) Q / G) holds iteration q
    return ((q + 1) * G - 1) // Q


def items(b, G, units, npair, kit):
    """The item sequence of CTA b: (unit, h, k0, k1, shared, slot)."""
    L = npair * kit
    dp = dp_units(units, G)
    Q = (units - dp) * L
    qb, qe = Q * b // G, Q * (b + 1) // G
    out = []
    u = b
    while u < dp:
        for h in range(npair):
            out.append((u, h, 0, kit, False, -1))
        u += G
    q = qb
    while q < qe:
        v = q // L
        r = q - v * L
        h = r // kit
        k0 = r - h * kit
        e = min(qe, v * L + (h + 1) * kit)
        k1 = k0 + (e - q)
        q = e
        shared = v * L < qb or (v + 1) * L > qe
        slot = 4 * b + (0 if v == qb // L else 2) + h
        out.append((dp + v, h, k0, k1, shared, slot))
    return out


def deliveries(unit, G, units, npair, kit):
    L = npair * kit
    dp = dp_units(units, G)
    Q = (units - dp) * L
    unit -= dp
    n = 0
    for h in range(npair):
        s = unit * L + h * kit
        e = s + kit
        for b in range(owner(Q, s, G), owner(Q, e - 1, G) + 1):
            if max(Q * b // G, s) < min(Q * (b + 1) // G, e):
                n += 1
    return n


def finisher_slots(unit, h, G, units, npair, kit):
    L = npair * kit
    dp = dp_units(units, G)
    Q = (units - dp) * L
    unit -= dp
    s = unit * L + h * kit
    e = s + kit
    out = []
    for b in range(owner(Q, s, G), owner(Q, e - 1, G) + 1):
        blo = Q * b // G
        if max(blo, s) >= min(Q * (b + 1) // G, e):
            continue
        out.append((b, 4 * b + (0 if unit == blo // L else 2) + h))
    return out


def check(G, units, npair, kit):
    cover = {}
    count, writers = {}, {}
    for b in range(G):
        for (u, h, k0, k1, shared, slot) in items(b, G, units, npair, kit):
            assert 0 <= k0 < k1 <= kit
            for k in range(k0, k1):
                assert (u, h, k) not in cover
                cover[(u, h, k)] = b
            if shared:
                assert 0 <= slot < 4 * G
                count[u] = count.get(u, 0) + 1
                writers.setdefault((u, h), []).append((b, slot))
    assert len(cover) == units * npair * kit
    for u in range(units):
        owners = {cover[(u, h, k)] for h in range(npair) for k in range(kit)}
        if len(owners) == 1:
            assert u not in count
            continue
        assert count[u] == deliveries(u, G, units, npair, kit)
        for h in range(npair):
            assert sorted(writers[(u, h)]) == finisher_slots(u, h, G, units, npair, kit)
    slots = [s for v in writers.values() for (_, s) in v]
    assert len(slots) == len(set(slots))
    per_cta = {}
    for (u, _), v in writers.items():
        for b, _ in v:
            per_cta.setdefault(b, set()).add(u)
    assert all(len(x) <= 2 for x in per_cta.values())


@pytest.mark.parametrize("G,units,npair,kit", [
    (152, 384, 1, 32),    # Schnakenberg 1024^2, F group mode 1 (2.5 waves)
    (152, 128, 1, 32),    # D group mode 1 (fewer units than CTAs)
    (152, 32, 2, 64),     # D group last mode, component pairs
    (152, 96, 2, 64),     # F group last mode
    (152, 1536, 1, 8),    # FHN 256^3 first mode (10 waves)
    (3, 7, 2, 1),         # one-chunk tiles
])
def test_schedule_of_benchmark_launches(G, units, npair, kit):
    check(G, units, npair, kit)


def test_schedule_random_shapes():
    rng = random.Random(1)
    for _ in range(400):
        npair = rng.choice([1, 2])
        kit = rng.randint(1, 70)
        units = rng.randint(1, 700)
        Q = units * npair * kit
        G = min(152, Q // 4) if rng.random() < 0.7 else rng.randint(2, 160)
        if G >= 2:
            check(G, units, npair, kit)
