"""Multi-rank host logic on CPU with gloo, world size 2: sharding of
independent systems, the max-over-ranks step time, a lost rank detected by a
short collective timeout (host-side fault injection; no GPU), and the
orbital-unit partition of one system: each rank's partial energies, V_avg
and gradients (formed by the oracle for its own orbitals, as the library's
orbital mask defines them) summed over the ranks equal the unsharded
oracle results."""
import multiprocessing as mp
import os
import socket

import pytest

from paper_2108_01186_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import torch.distributed as dist
        timeout = 5 if mode == "lost" else 60
        D.init("gloo", timeout_s=timeout)
        if mode == "ok":
            units = D.shard(64, rank, world)
            t = D.max_over_ranks(10.0 + rank)
            D.barrier()
            q.put((rank, units, t))
        elif mode == "orbitals":
            q.put((rank, "orbitals", _orbital_partials(rank, world)))
        else:
            if rank == 1:
                q.put((rank, "left", None))
                q.close()
                q.join_thread()        # the message is out before the process dies
                os._exit(0)            # leaves between steps, nothing in flight
            try:
                D.max_over_ranks(1.0)
                q.put((rank, "no error", None))
            except Exception as e:     # the collective ends with an error
                q.put((rank, "error", type(e).__name__))
        dist.destroy_process_group() if dist.is_initialized() and mode == "ok" else None
    except Exception as e:
        q.put((rank, "exception", repr(e)))


def _orbital_partials(rank, world):
    """This rank's share of one system's step, reduced over the ranks."""
    import numpy as np
    import torch
    import oracle
    from paper_2108_01186_gb300 import synth
    oracle.build_library()
    s = synth.make_system(20, 0.45, 2, [3, 2], seed=31)
    ref = oracle.sic_forward(s.psi, s.fods, s.grid, scale=0.5, tol=1e-12)
    norb = sum(s.norb)
    mask = np.array(D.orbital_mask(norb, rank, world))
    dV = s.h ** 3
    Vavg, U, X, E = [], [], [], 0.0
    fwd = dict(blocks=[], E_sic=0.0)
    off = 0
    for sp, b in enumerate(ref["blocks"]):
        m = mask[off:off + len(b["U"])]
        rho_s = np.sum(s.psi[sp] ** 2, axis=0)
        num = np.sum((m[:, None] * b["rho"]) * -(b["V"] + b["vxc"]), axis=0)
        Vavg.append(np.where(rho_s > 1e-30, 0.5 * num / np.where(rho_s > 1e-30, rho_s, 1.0), 0.0))
        U.append(m * b["U"])
        X.append(m * b["Exc"])
        E -= float(np.sum(m * (b["U"] + b["Exc"])))
        # the masked orbitals' adjoint seeds vanish: V^SIC = -(V + v_xc) = 0
        bb = dict(b)
        bb["V"] = np.where(m[:, None] == 1, b["V"], -b["vxc"])
        bb.update(psi=s.psi[sp], fods=s.fods[sp])
        fwd["blocks"].append(bb)
        off += len(b["U"])
    dpsi, dfod = oracle.sic_backward(fwd, s.grid, tol=1e-12)
    parts = [torch.tensor(np.concatenate(Vavg)), torch.tensor(np.concatenate(U)), torch.tensor(np.concatenate(X)),
             torch.tensor([E], dtype=torch.float64), torch.tensor(np.concatenate([d.ravel() for d in dpsi])),
             torch.tensor(np.concatenate([d.ravel() for d in dfod]))]
    D.allreduce_sum(parts)
    # the unsharded reference
    full_dpsi, full_dfod = oracle.sic_backward(dict(blocks=[dict(b, psi=s.psi[k], fods=s.fods[k])
                                                            for k, b in enumerate(ref["blocks"])], E_sic=0.0),
                                               s.grid, tol=1e-12)
    want = [np.concatenate([b["Vavg"] for b in ref["blocks"]]), np.concatenate([b["U"] for b in ref["blocks"]]),
            np.concatenate([b["Exc"] for b in ref["blocks"]]), np.array([ref["E_sic"]]),
            np.concatenate([d.ravel() for d in full_dpsi]), np.concatenate([d.ravel() for d in full_dfod])]
    return int(mask.sum()), [float(np.max(np.abs(p.numpy() - w)) / max(1.0, np.max(np.abs(w))))
                             for p, w in zip(parts, want)]


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return sorted(out, key=lambda x: x[0])


def test_shard_covers_every_unit_once():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            got = [u for r in range(world) for u in D.shard(n, r, world)]
            assert got == list(range(n))
            sizes = [len(D.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.shard(4, 2, 2)


def test_two_gloo_ranks_shard_and_max_time():
    out = _run("ok")
    assert out[0][1] + out[1][1] == list(range(64))
    assert out[0][2] == 11.0 and out[1][2] == 11.0


def test_lost_rank_is_detected_by_collective_timeout():
    out = _run("lost")
    assert out[1][1] == "left"
    assert out[0][1] == "error"


def test_two_gloo_ranks_orbital_partition_sums_to_the_whole():
    out = _run("orbitals")
    assert [o[1] for o in out] == ["orbitals", "orbitals"], out
    counts = [o[2][0] for o in out]
    assert sorted(counts) == [2, 3]                      # 5 orbitals split 3 + 2
    for _, _, (n, errs) in out:
        # V_avg, U, E_xc, E_SIC, dE/dpsi, dE/da: partial sums over the ranks equal the whole
        assert max(errs) < 1e-12, errs


def test_orbital_mask_partitions_every_orbital_once():
    for norb in (1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            masks = [D.orbital_mask(norb, r, world) for r in range(world)]
            assert all(sum(m[o] for m in masks) == 1 for o in range(norb))
