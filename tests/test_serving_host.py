"""Host logic of the serving loop: slot admission under a memory budget."""
from paper_2603_01122_gb300.serving import SlotTable


def test_slots_and_budget():
    st = SlotTable(capacity=4, budget_bytes=3 * 100, slot_bytes=100)
    a = [st.admit(k) for k in "abcd"]
    assert a[:3] == [0, 1, 2] and a[3] is None          # the budget binds before the slots
    st.retire(1)
    assert st.admit("e") == 1                          # the freed slot is reused
    assert st.used_bytes == 300 and not st.can_admit()
    st.retire(0)
    st.retire(2)
    assert st.admit("f") == 0 and st.admit("g") == 2
    assert set(st.live.values()) == {"e", "f", "g"}


def test_capacity_binds_when_budget_is_large():
    st = SlotTable(capacity=2, budget_bytes=1 << 40, slot_bytes=10)
    assert st.admit(1) == 0 and st.admit(2) == 1 and st.admit(3) is None
