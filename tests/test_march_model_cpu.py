"""CPU model of the z-march bookkeeping of the staged complex FP32 sweep (k_zsweep_sm): the march
is unrolled by the z-queue length Q = 2r + 1, plane z + d lives in register slot (u + r + d) mod Q
at step z = zb + u (zb - z0 a multiple of Q), the plane loaded one step ahead (z + 1 + r) replaces
the slot of the plane that left, and the staged in-plane buffers turn with a counter (buffer of
plane z: (z - z0) mod 3, fill of plane z + 2 into the buffer of plane z - 1). The model replays the
kernel's index arithmetic on plane labels and checks every read against a plain shifting queue,
for every radius, ragged z ranges and periodic wrap (no GPU needed).
"""
import pytest

NBUF = 3


def wrap(j, n):
    q = j % n
    return q + n if q < 0 else q


def plane_value(jz, nz, periodic):
    # the label the kernel would load for plane jz: its wrapped index, or None (a zero ghost)
    if periodic:
        return wrap(jz, nz)
    return jz if 0 <= jz < nz else None


def run_unrolled(r, z0, z1, nz, periodic):
    """The kernel's march: returns, per step, the z column it reads (planes z - r .. z + r) and the
    staged buffer it reads the in-plane neighbours from, plus the buffer each fill writes."""
    Q = 2 * r + 1
    q = [plane_value(z0 + k - r, nz, periodic) for k in range(Q)]  # initial queue, slot k = plane z0 + k - r
    staged = {0: z0, 1: z0 + 1}  # fill(z0, 0), fill(z0 + 1, 1)
    qn = None
    buf = 0
    reads = []
    zb = z0
    while zb < z1:
        for u in range(Q):
            z = zb + u
            if z >= z1:
                break
            staged[NBUF - 1 if buf == 0 else buf - 1] = z + 2  # fill(z + 2, ...): the buffer of plane z - 1
            if u > 0 or zb > z0:
                q[(u + Q - 1) % Q] = qn
            if z + 1 < z1:
                jz = z + 1 + r
                qn = (jz if jz < nz else wrap(jz, nz)) if periodic else (jz if jz < nz else None)
            col = [q[(u + r + d) % Q] for d in range(-r, r + 1)]
            assert staged[buf] == z, (z, buf, staged)  # the in-plane neighbours come from plane z
            reads.append((z, col))
            buf = 0 if buf == NBUF - 1 else buf + 1
        zb += Q
    return reads


def run_shifting(r, z0, z1, nz, periodic):
    """The plain form: a queue of 2r + 1 planes shifted by one every step."""
    Q = 2 * r + 1
    q = [plane_value(z0 + k - r, nz, periodic) for k in range(Q)]
    reads = []
    for z in range(z0, z1):
        if z > z0:
            q = q[1:] + [plane_value(z + r, nz, periodic)]
        reads.append((z, list(q)))
    return reads


@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("periodic", [False, True])
def test_unrolled_march_reads_the_same_planes(r, periodic):
    Q = 2 * r + 1
    for nz in (1, 2, Q - 1, Q, Q + 1, 3 * Q + 2, 40):
        for zc in (1, 2, Q - 1, Q, Q + 1, 2 * Q + 3, 16):
            for z0 in range(0, nz, zc):
                z1 = min(nz, z0 + zc)
                got = run_unrolled(r, z0, z1, nz, periodic)
                want = run_shifting(r, z0, z1, nz, periodic)
                assert got == want, (r, periodic, nz, zc, z0)
                # and the column really is planes z - r .. z + r
                for z, col in want:
                    assert col == [plane_value(z + d, nz, periodic) for d in range(-r, r + 1)]


def test_model_catches_a_wrong_slot():
    # a plausible slip (the entering plane written to slot u instead of u - 1) must be caught
    r, z0, z1, nz = 3, 0, 20, 20
    Q = 2 * r + 1
    q = [plane_value(z0 + k - r, nz, False) for k in range(Q)]
    qn, bad = None, False
    for zb in range(z0, z1, Q):
        for u in range(Q):
            z = zb + u
            if z >= z1:
                break
            if u > 0 or zb > z0:
                q[u % Q] = qn
            if z + 1 < z1:
                jz = z + 1 + r
                qn = jz if jz < nz else None
            col = [q[(u + r + d) % Q] for d in range(-r, r + 1)]
            if col != [plane_value(z + d, nz, False) for d in range(-r, r + 1)]:
                bad = True
    assert bad
