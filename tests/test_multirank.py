"""Multi-process logic of bench.py on CPU ranks (gloo, world size 2): the
barrier, the max-over-ranks time and the weak-scaling aggregate.  The data
path has no collective (each rank reconstructs its own slice), so this is the
only cross-rank code."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_dist_barrier_max_and_weak_aggregate(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent(f"""
        import os, sys, json
        sys.path.insert(0, {ROOT!r})
        import bench
        d = bench.Dist()
        d.barrier()
        ms = 10.0 + 5.0 * d.rank            # rank 1 is slower
        worst = d.max(ms)
        steps = 4
        value = d.world * 1000.0 * steps / worst
        d.barrier()
        print(json.dumps({{"rank": d.rank, "world": d.world, "worst": worst, "value": value}}))
        d.close()
    """))
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()), CUDA_VISIBLE_DEVICES="")
    procs = []
    for r in range(2):
        e = dict(env, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2")
        procs.append(subprocess.Popen([sys.executable, str(script)], env=e, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    import json
    res = [json.loads(o[0].strip().splitlines()[-1]) for o in outs]
    assert all(p.returncode == 0 for p in procs), [o[1] for o in outs]
    for r in res:
        assert r["world"] == 2 and r["worst"] == 15.0
        assert abs(r["value"] - 2 * 1000.0 * 4 / 15.0) < 1e-9


def test_reference_arm_other_ranks_exit_quietly(tmp_path):
    script = tmp_path / "ref.py"
    script.write_text(textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        import bench
        class A: pass
        a = A(); a.gpus = 2; a.steps = 1; a.warmup = 0
        class D: rank = 1
        bench.run_reference(a, D())          # non-zero rank: no work, no output
        print("ok")
    """))
    out = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip() == "ok"
