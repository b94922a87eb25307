"""Element partitions (paper_2408_06698_gb300/partition.py), on the CPU.

* the facet neighbours found from representative vertex tuples are the oracle topology's;
* slab partitions own every element once, their halo is exactly the facet neighbours owned
  elsewhere, and each send list matches the receiving partition's halo order;
* the oracle's apply on every partition's local mesh, with the halo filled from the owners,
  equals the oracle's apply on the whole mesh on the owned elements, bit for bit;
* the same exchange plan run between two CPU ranks (torch.distributed, gloo) fills each
  rank's halo with the owners' blocks, and the rank's oracle apply then matches.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh
from paper_2408_06698_gb300.partition import facet_neighbours, partitions_from_owner, slab_partitions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("dim,n,periodic", [(3, 3, True), (3, 3, False), (2, 5, True)])
def test_facet_neighbours_match_the_oracle_topology(dim, n, periodic):
    m = W.periodic_box_mesh(dim, n)
    rep = m.rep if periodic else None
    nb = facet_neighbours(m.elems, rep)
    topo = mesh.MeshTopo(m.coords, m.elems, rep)
    # the oracle sorts each element's vertices by representative: local facet f of the
    # oracle is opposite its sorted vertex f; compare as sets of neighbours per element
    for e in range(m.n_elems):
        mine = sorted(int(x) for x in nb[e])
        ref = []
        for F in topo.elem_facet[e]:
            other = topo.fb[F, 0] if topo.fa[F, 0] == e else topo.fa[F, 0]
            ref.append(int(other))
        assert mine == sorted(ref), e


@pytest.mark.parametrize("dim,n,P", [(3, 4, 2), (3, 4, 3), (2, 6, 4)])
def test_slab_partitions_and_exchange_plan(dim, n, P):
    m = W.periodic_box_mesh(dim, n)
    parts = slab_partitions(m, P)
    owned = np.concatenate([p.owned for p in parts])
    assert np.array_equal(np.sort(owned), np.arange(m.n_elems))
    nb = facet_neighbours(m.elems, m.rep)
    owner = np.empty(m.n_elems, dtype=np.int64)
    for p in parts:
        owner[p.owned] = p.rank
    for p in parts:
        want = np.unique(nb[p.owned].reshape(-1))
        want = want[owner[want] != p.rank]
        assert np.array_equal(np.sort(p.halo), want)
        for q, idx in p.recv.items():
            g_recv = p.local[idx]
            g_send = parts[q].local[parts[q].send[p.rank]]
            assert np.array_equal(g_recv, g_send) and np.all(owner[g_recv] == q)
            assert np.all(parts[q].send[p.rank] < parts[q].n_owned)


def _oracle_partitioned(m, parts, k, l, seed=3):
    topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
    ref = fe.ref_element(m.dim, k)
    sp = hdiv.HDiv(topo, ref)
    rng = np.random.default_rng(seed)
    wL = sp.to_l2(rng.standard_normal(sp.n_hdiv))
    uL = rng.standard_normal((topo.n_elems, m.dim, ref.nb))
    full = C.apply(topo, ref, wL, uL, l)
    return topo, ref, wL, uL, full


@pytest.mark.parametrize("dim,n,k,P", [(3, 4, 2, 3), (2, 6, 3, 2)])
def test_partitioned_oracle_apply_equals_whole_mesh(dim, n, k, P):
    m = W.periodic_box_mesh(dim, n)
    parts = slab_partitions(m, P)
    topo, ref, wL, uL, full = _oracle_partitioned(m, parts, k, k - 1)
    for p in parts:
        sub = mesh.MeshTopo(m.coords, m.elems[p.local], m.rep)
        y = C.apply(sub, ref, wL[p.local], uL[p.local], k - 1)
        assert np.array_equal(y[: p.n_owned], full[p.owned])


def test_owner_partitions_need_not_be_slabs():
    m = W.periodic_box_mesh(3, 3)
    owner = np.random.default_rng(0).integers(0, 3, size=m.n_elems)
    owner[:3] = [0, 1, 2]
    parts = partitions_from_owner(m.elems, m.rep, owner)
    topo, ref, wL, uL, full = _oracle_partitioned(m, parts, 2, 1)
    for p in parts:
        sub = mesh.MeshTopo(m.coords, m.elems[p.local], m.rep)
        y = C.apply(sub, ref, wL[p.local], uL[p.local], 1)
        assert np.array_equal(y[: p.n_owned], full[p.owned])


_RANK_SCRIPT = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
import workloads as W
from oracle import convection as C
from oracle import fe, hdiv, mesh
from paper_2408_06698_gb300.partition import slab_partitions, exchange_host
rank = int(os.environ["RANK"]); world = int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
dim, n, k = 3, 4, 2
m = W.periodic_box_mesh(dim, n)
parts = slab_partitions(m, world)
part = parts[rank]
topo = mesh.MeshTopo(m.coords, m.elems, m.rep)
ref = fe.ref_element(dim, k)
sp = hdiv.HDiv(topo, ref)
rng = np.random.default_rng(5)                         # every rank draws the same global fields
wL = sp.to_l2(rng.standard_normal(sp.n_hdiv))
uL = rng.standard_normal((topo.n_elems, dim, ref.nb))
nloc = dim * ref.nb
loc_u = np.zeros((len(part.local), nloc)); loc_u[: part.n_owned] = uL[part.owned].reshape(-1, nloc)
loc_w = np.zeros((len(part.local), nloc)); loc_w[: part.n_owned] = wL[part.owned].reshape(-1, nloc)
exchange_host(part, loc_u, nloc)
exchange_host(part, loc_w, nloc)
halo_ok = bool(np.array_equal(loc_u, uL[part.local].reshape(-1, nloc)) and
               np.array_equal(loc_w, wL[part.local].reshape(-1, nloc)))
sub = mesh.MeshTopo(m.coords, m.elems[part.local], m.rep)
y = C.apply(sub, ref, loc_w.reshape(-1, dim, ref.nb), loc_u.reshape(-1, dim, ref.nb), k - 1)
full = C.apply(topo, ref, wL, uL, k - 1)
apply_ok = bool(np.array_equal(y[: part.n_owned], full[part.owned]))
print(json.dumps({{"rank": rank, "halo_ok": halo_ok, "apply_ok": apply_ok, "halo": int(len(part.halo))}}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_halo_exchange_between_two_cpu_ranks(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(_RANK_SCRIPT.format(root=ROOT))
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    assert all(p.returncode == 0 for p in procs), outs
    res = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    assert all(r["halo_ok"] and r["apply_ok"] and r["halo"] > 0 for r in res), res
