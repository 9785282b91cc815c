"""FP64 CPU oracle of the QEq path and of the warm-start network: TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of bench.py may import it;
it shares no code with the CUDA path (only the seeded input generators are common to both).
"""
