"""T_s search (Sec. III.B) with batched GPU solves against the same search on oracle solves
(the XY algorithm from the sector ground state of H^xy on both sides, Sec. III.A.3)."""
import pytest

from instances import generate_ec3
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_3938_gb300 as P

    P.build()
    yield


@pytest.mark.parametrize("driver", ["x", "xy"])
def test_batched_Ts_matches_oracle(driver):
    from paper_1311_3938_gb300 import _native as N
    from paper_1311_3938_gb300 import hamiltonians as HB
    from paper_1311_3938_gb300.tsearch import gpu_energies, search_Ts
    from paper_1311_3938_gb300.workloads import Job

    n, seed = 8, 3
    inst = generate_ec3(n, seed)
    job = Job(jid=0, n=n, seed=seed, nonlinear=False, T=1.0, precision=N.AQC_C128, driver=driver)
    r_gpu = search_Ts(gpu_energies(job), 1.0, 64.0, k=8, rtol=1e-3)
    if driver == "x":
        H = O.ec3_hamiltonian(inst)
        psi0 = O.uniform_state(n)
    else:
        H = O.xy_hamiltonian(inst, driver="xy")
        psi0 = O.xy_sector_ground_state(n, inst.clauses, bin(inst.solution).count("1"))[1]

    def E(Ts):
        out = []
        for T in Ts:
            sched = O.linear_path(T)
            res = O.propagate(H, sched, O.step_count(H, sched), psi0)
            out.append(O.energy(H, res.psi, 1))
        return out

    r_or = search_Ts(E, 1.0, 64.0, k=8, rtol=1e-3)
    assert r_gpu["Ts"] is not None and r_or["Ts"] is not None
    assert abs(r_gpu["Ts"] / r_or["Ts"] - 1.0) < 1e-6
