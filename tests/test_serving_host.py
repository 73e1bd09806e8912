"""Host logic of the serving loop: slot admission under a memory budget, and
the detection of a human leaving a goal."""
from paper_2603_01122_gb300.serving import GoalDeparture, SlotTable


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


def test_goal_departure():
    d = GoalDeparture([[0.0, 0.0], [5.0, 5.0]], radius=0.5)
    path = [(2.0, 2.0), (0.9, 0.2), (0.3, 0.1), (0.1, 0.0), (0.45, 0.0), (0.6, 0.0), (1.0, 0.0),
            (4.7, 4.9), (5.0, 5.0), (6.0, 5.0)]
    got = [d.update(p) for p in path]
    # arriving, staying and moving inside the radius are not departures; the
    # first state beyond every goal's radius after being near one is
    assert got == [False, False, False, False, False, True, False, False, False, True]
